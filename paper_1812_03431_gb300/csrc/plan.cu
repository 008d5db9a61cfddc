// Plan creation for librexi: Gaussian grid and Legendre tables (Sec. 3), REXI
// poles (Sec. 4.1), the per-(pole, m, n) factors of the banded solves (Sec. 5)
// for the step and its adjoint, solve work lists and workspaces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>

#include "rexi_internal.h"

namespace rexi {

bool fft_factor(int n, int *radix, int *nstages);
cudaError_t fft_configure(Plan &pl);
cudaError_t legendre_configure();
cudaError_t tc_setup(Plan &pl);

namespace {

template <typename T>
cudaError_t upload(T **dev, const std::vector<T> &host, size_t *bytes) {
  cudaError_t e = cudaMalloc(dev, std::max<size_t>(1, host.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  *bytes += host.size() * sizeof(T);
  if (host.empty()) return cudaSuccess;
  return cudaMemcpy(*dev, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
cudaError_t dalloc(T **dev, size_t count, size_t *bytes) {
  cudaError_t e = cudaMalloc(dev, std::max<size_t>(1, count) * sizeof(T));
  if (e == cudaSuccess) *bytes += count * sizeof(T);
  return e;
}

double eps_nm(int n, int m) {
  if (n <= m) return 0.0;
  return std::sqrt(((double)n * n - (double)m * m) / (4.0 * n * n - 1.0));
}

// Pole-independent zeta weights W_n = sum_k beta_k / (alpha_k + i tau sigma_n) and the
// adjoint's sum_k conj(beta_k) / (conj(alpha_k) - i tau sigma_n); zero for rows that
// are not state (zeta_0^0).
__global__ void zeta_weights_kernel(const double *coef, const int32_t *m_of, const double2 *alpha,
                                    const double2 *beta, int P, int64_t NS, double tau, double2 *wf, double2 *wa) {
  const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= NS) return;
  const double sig = coef[4 * ix + 0];
  const double G = coef[4 * ix + 3];  // n (n + 1) / a^2, zero only at n = 0
  double2 sf = make_double2(0, 0), sa = make_double2(0, 0);
  if (G > 0.0 || m_of[ix] > 0) {
    for (int k = 0; k < P; ++k) {
      const double2 al = alpha[k], be = beta[k];
      // beta / (alpha + i tau sigma)
      double dr = al.x, di = al.y + tau * sig, d = dr * dr + di * di;
      sf.x += (be.x * dr + be.y * di) / d;
      sf.y += (be.y * dr - be.x * di) / d;
      // conj(beta) / (conj(alpha) - i tau sigma)
      dr = al.x;
      di = -al.y - tau * sig;
      d = dr * dr + di * di;
      sa.x += (be.x * dr - be.y * di) / d;
      sa.y += (-be.y * dr - be.x * di) / d;
    }
  }
  wf[ix] = sf;
  wa[ix] = sa;
}

// Orthonormal Pbar_n^m(mu_j) and H_n^m(mu_j) for the northern latitudes j < J, one
// thread per (m, j): the m-diagonal seed and the three-term recurrence in n (the same
// recurrences as the oracle's tables, written independently).  Layout [idx(m, n)][J].
__global__ void alp_tables_kernel(const double *mu_all, int N, int J, double *tabP, double *tabH) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(N + 1) * J) return;
  const int m = (int)(t / J), j = (int)(t - (int64_t)m * J);
  const double mu = mu_all[j];
  const double s = sqrt(1.0 - mu * mu);
  double pmm = 1.0 / sqrt(2.0);
  for (int k = 1; k <= m; ++k) pmm *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
  const int64_t idx0 = (int64_t)m * (2 * N + 3 - m) / 2;
  auto eps = [m](int n) { return n <= m ? 0.0 : sqrt(((double)n * n - (double)m * m) / (4.0 * n * n - 1.0)); };
  // p_{n-1}, p_n, p_{n+1} rolling; H_n needs p_{n-1} and p_{n+1}
  double pm1 = 0.0, p0 = pmm;
  double p1 = sqrt(2.0 * m + 3.0) * mu * pmm;  // degree m + 1
  for (int n = m; n <= N; ++n) {
    const double h = -n * eps(n + 1) * p1 + (n > m ? (n + 1) * eps(n) * pm1 : 0.0);
    tabP[(idx0 + n - m) * J + j] = p0;
    tabH[(idx0 + n - m) * J + j] = h;
    const double p2 = (mu * p1 - eps(n + 1) * p0) / eps(n + 2);  // degree n + 2
    pm1 = p0;
    p0 = p1;
    p1 = p2;
  }
}

}  // namespace

void free_plan(Plan *pl);

rexi_status build_plan(const rexi_params &prm, Plan *pl) {
  pl->prm = prm;
  pl->ff = prm.solve_arith == REXI_SOLVE_FP32X2;
  pl->ffil = pl->ff && prm.max_batch >= 8;
  const int N = prm.ntrunc;
  pl->N = N;
  pl->nlat = prm.nlat;
  pl->nlon = prm.nlon;
  pl->J = prm.nlat / 2;
  pl->nspec = nspec_of(N);
  size_t &bytes = pl->bytes;
  cudaError_t e;
  auto fail = [&](const char *what, cudaError_t err) {
    set_error(std::string("plan: ") + what + ": " + cudaGetErrorString(err));
    return err == cudaErrorMemoryAllocation ? REXI_ENOMEM : REXI_ECUDA;
  };
  cudaGetDevice(&pl->device);
  cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);

  // device error word (rexi_check_device; the float-float factor split below reports to it)
  if ((e = dalloc(&pl->dev_err, 1, &bytes))) return fail("error word", e);
  if ((e = cudaMemset(pl->dev_err, 0, sizeof(int)))) return fail("error word", e);

  // ---- poles
  if (prm.alpha && prm.beta) {
    pl->P = prm.npoles;
    pl->alpha.resize(pl->P);
    pl->beta.resize(pl->P);
    for (int k = 0; k < pl->P; ++k) {
      pl->alpha[k] = cplx(prm.alpha[2 * k], prm.alpha[2 * k + 1]);
      pl->beta[k] = cplx(prm.beta[2 * k], prm.beta[2 * k + 1]);
    }
  } else {
    rexi_coeffs_host(prm.M, prm.h, prm.normalize != 0, pl->alpha, pl->beta, &pl->eps0);
    pl->P = (int)pl->alpha.size();
  }
  if (prm.pole_begin != 0 || prm.pole_end != 0) {  // this plan's share of the poles
    if (prm.pole_begin < 0 || prm.pole_end <= prm.pole_begin || prm.pole_end > pl->P) {
      set_error("plan: need 0 <= pole_begin < pole_end <= P (P = " + std::to_string(pl->P) + ")");
      return REXI_EINVAL;
    }
    pl->alpha = std::vector<cplx>(pl->alpha.begin() + prm.pole_begin, pl->alpha.begin() + prm.pole_end);
    pl->beta = std::vector<cplx>(pl->beta.begin() + prm.pole_begin, pl->beta.begin() + prm.pole_end);
    pl->P = prm.pole_end - prm.pole_begin;
  }
  const int P = pl->P;
  const double tau = prm.tau, a = prm.radius, om = prm.omega;
  const double phibar = prm.gravity * prm.mean_depth;
  if (prm.strict_range) {
    const double wmax = std::sqrt(4.0 * om * om + phibar * N * (N + 1.0) / (a * a));
    if (tau * wmax > prm.h * (prm.M - 10)) {
      set_error("plan: tau * max|omega| exceeds h (M - 10)");
      return REXI_ERANGE;
    }
  }
  std::vector<double2> al(P), be(P);
  for (int k = 0; k < P; ++k) {
    al[k] = make_double2(pl->alpha[k].real(), pl->alpha[k].imag());
    be[k] = make_double2(pl->beta[k].real(), pl->beta[k].imag());
  }
  if ((e = upload(&pl->alpha_dev, al, &bytes))) return fail("alpha", e);
  if ((e = upload(&pl->beta_dev, be, &bytes))) return fail("beta", e);

  // ---- systems (m, parity) and rows: delta rows (n >= max(m, 1)) for the delta
  // elimination, Phi rows (n >= m, Phi_0^0 included) for the geopotential-only solver
  const bool phi_solver = prm.solver == REXI_SOLVER_PHI;
  pl->sys.resize(2 * (N + 1));
  int64_t row = 0;
  int lmax = 0;
  for (int m = 0; m <= N; ++m)
    for (int p = 0; p < 2; ++p) {
      const int nmin = phi_solver ? m : std::max(m, 1);
      int n0 = m + p;
      while (n0 < nmin) n0 += 2;
      const int len = n0 <= N ? (N - n0) / 2 + 1 : 0;
      pl->sys[2 * m + p] = SysInfo{m, p, n0, len, row};
      row += len;
      lmax = std::max(lmax, len);
    }
  pl->nrows = row;
  pl->lmax = std::max(lmax, 1);
  std::vector<int4> sysv;
  for (const SysInfo &s : pl->sys) sysv.push_back(make_int4(s.m, s.n0, s.len, (int)s.row0));
  if ((e = upload(&pl->sys_dev, sysv, &bytes))) return fail("systems", e);

  // ---- per-coefficient data: sigma, ct, dt, G; zonal order; reduce flags; zeta weights
  const int64_t NS = pl->nspec;
  std::vector<double> coef(4 * NS, 0.0);
  std::vector<int32_t> m_of(NS);
  std::vector<uint8_t> rflags(3 * NS, 0);
  std::vector<double> zd_syn(NS), zd_ana_adj(NS), zd_one(NS, 1.0), zd_mone(NS, -1.0);
  for (int m = 0; m <= N; ++m) {
    const int nmin = std::max(m, 1);
    for (int n = m; n <= N; ++n) {
      const int64_t ix = spec_idx(N, m, n);
      m_of[ix] = m;
      double sig = 0, ct = 0, dt = 0;
      if (n > 0) {
        sig = 2.0 * om * m / (n * (n + 1.0));
        if (n - 1 >= nmin) ct = eps_nm(n, m) * (n + 1.0) / n;
        if (n + 1 <= N) dt = eps_nm(n + 1, m) * n / (n + 1.0);
      }
      coef[4 * ix + 0] = sig;
      coef[4 * ix + 1] = ct;
      coef[4 * ix + 2] = dt;
      coef[4 * ix + 3] = n * (n + 1.0) / (a * a);
      zd_syn[ix] = n > 0 ? -a / (n * (n + 1.0)) : 0.0;
      zd_ana_adj[ix] = n > 0 ? a / (n * (n + 1.0)) : 0.0;
      // reduce flags: Phi/delta rows have partials iff n >= nmin; zeta rows iff a
      // delta row of the other parity sits at n - 1 or n + 1
      const bool staterow = n >= nmin;
      if (!phi_solver) {
        rflags[0 * NS + ix] = staterow ? 1 : 0;
        rflags[2 * NS + ix] = staterow ? 1 : 2;
        bool zp = staterow && ((n - 1 >= nmin) || (n + 1 <= N));
        rflags[1 * NS + ix] = staterow ? (zp ? 1 : 0) : 2;
      } else {
        // every Phi row is solved; zeta rows collect from Phi rows at n -+ 1 of the
        // other parity; zeta_0^0 and delta_0^0 are not state
        rflags[0 * NS + ix] = 1;
        rflags[2 * NS + ix] = staterow ? 1 : 2;
        rflags[1 * NS + ix] = staterow ? (((n - 1 >= m) || (n + 1 <= N)) ? 1 : 0) : 2;
      }
    }
  }
  cplx sphf(0, 0), spha(0, 0);
  for (int k = 0; k < P; ++k) {
    sphf += pl->beta[k] / pl->alpha[k];
    spha += std::conj(pl->beta[k]) / std::conj(pl->alpha[k]);
  }
  pl->sphi_fwd = make_double2(sphf.real(), sphf.imag());
  pl->sphi_adj = make_double2(spha.real(), spha.imag());
  {
    cplx sb(0, 0);
    for (int k = 0; k < P; ++k) sb += pl->beta[k];
    pl->sumb = make_double2(sb.real(), sb.imag());
  }
  if ((e = upload(&pl->coef_dev, coef, &bytes))) return fail("coef", e);
  if ((e = upload(&pl->m_of_dev, m_of, &bytes))) return fail("m_of", e);
  if ((e = upload(&pl->rflags_dev, rflags, &bytes))) return fail("rflags", e);
  if ((e = dalloc(&pl->w_fwd, NS, &bytes))) return fail("w", e);
  if ((e = dalloc(&pl->w_adj, NS, &bytes))) return fail("w", e);
  zeta_weights_kernel<<<(unsigned)((NS + 127) / 128), 128>>>(pl->coef_dev, pl->m_of_dev, pl->alpha_dev,
                                                             pl->beta_dev, P, NS, tau, pl->w_fwd, pl->w_adj);
  if ((e = cudaGetLastError())) return fail("zeta weights", e);
  if ((e = upload(&pl->zd_syn, zd_syn, &bytes))) return fail("zd", e);
  if ((e = upload(&pl->zd_ana_adj, zd_ana_adj, &bytes))) return fail("zd", e);
  if ((e = upload(&pl->zd_one, zd_one, &bytes))) return fail("zd", e);
  if ((e = upload(&pl->zd_mone, zd_mone, &bytes))) return fail("zd", e);

  // ---- solve factors (forward now; adjoint on first use); the f-sphere needs none
  if (phi_solver) {
    // Galerkin matrices of mu^2, mu^4 and mu (1 - mu^2) d/dmu in orthonormal Legendre
    // functions, by the recurrences mu P_n = eps_{n+1} P_{n+1} + eps_n P_{n-1} and
    // (1 - mu^2) P_n' = -n eps_{n+1} P_{n+1} + (n + 1) eps_n P_{n-1}; products are taken
    // over all degrees and truncated afterwards (exact projection)
    std::vector<double> zc(12 * NS, 0.0);
    for (int m = 0; m <= N; ++m) {
      auto ep = [m](int k) { return k > m ? eps_nm(k, m) : 0.0; };
      auto mu2 = [&](int k, int d) {  // (mu^2)[k][k + 2d], d in -1..1
        if (d == -1) return ep(k) * ep(k - 1);
        if (d == 0) return ep(k) * ep(k) + ep(k + 1) * ep(k + 1);
        return ep(k + 1) * ep(k + 2);
      };
      for (int n = m; n <= N; ++n) {
        double *z = &zc[12 * spec_idx(N, m, n)];
        for (int d = -1; d <= 1; ++d) z[1 + d] = mu2(n, d);
        for (int d = -2; d <= 2; ++d) {  // (mu^4)[n][n + 2d] = sum_l mu2[n][l] mu2[l][n + 2d]
          double acc = 0.0;
          for (int d1 = -1; d1 <= 1; ++d1) {
            const int l = n + 2 * d1, d2 = d - d1;
            if (l < m || d2 < -1 || d2 > 1) continue;
            acc += mu2(n, d1) * mu2(l, d2);
          }
          z[5 + d] = acc;
        }
        z[8] = ep(n) * (-(n - 2.0) * ep(n - 1));
        z[9] = (n + 1.0) * ep(n) * ep(n) - n * ep(n + 1) * ep(n + 1);
        z[10] = ep(n + 1) * (n + 3.0) * ep(n + 2);
      }
    }
    if ((e = upload(&pl->phi_zc, zc, &bytes))) return fail("phi coefficients", e);
    const size_t nfac = (size_t)7 * pl->nrows * P;
    if ((e = dalloc(&pl->fac_fwd, nfac, &bytes))) return fail("factors", e);
    if ((e = launch_phi_factor(*pl, 0))) return fail("factor setup", e);
    if (pl->ff) {
      const rexi_status r = take_range_error(*pl, "plan: float-float factors");
      if (r != REXI_OK) return r;
    }
    if ((e = dalloc(&pl->phi_q, (size_t)5 * NS * prm.max_batch, &bytes))) return fail("phi rhs", e);
    if (pl->ff) {  // alpha, beta and beta alpha as float-float values (hi = fl32(x), lo = fl32(x - hi))
      auto split = [](double x) {
        const float hi = (float)x;
        return std::make_pair(hi, (float)(x - (double)hi));
      };
      std::vector<float4> abf(3 * (size_t)P);
      for (int k = 0; k < P; ++k) {
        const cplx v[3] = {pl->alpha[k], pl->beta[k], pl->beta[k] * pl->alpha[k]};
        for (int j = 0; j < 3; ++j) {
          const auto re = split(v[j].real()), im = split(v[j].imag());
          abf[(size_t)j * P + k] = make_float4(re.first, re.second, im.first, im.second);
        }
      }
      float4 *d = nullptr;
      if ((e = upload(&d, abf, &bytes))) return fail("phi poles", e);
      pl->phi_abf = reinterpret_cast<double2 *>(d);
    }
  } else if (!prm.fsphere) {
    if (pl->ff) {  // compact float-float factors: tau G_n per idx and 1/alpha per pole
      auto split = [](double x) { const float hi = (float)x; return make_float2(hi, (float)(x - (double)hi)); };
      std::vector<float2> rows((size_t)NS);
      for (int m = 0; m <= N; ++m)
        for (int n = m; n <= N; ++n)
          rows[(size_t)spec_idx(N, m, n)] = split(tau * (double)n * (n + 1.0) / (a * a));
      std::vector<float4> ia((size_t)P);
      for (int k = 0; k < P; ++k) {
        const cplx v = 1.0 / pl->alpha[k];
        const float2 re = split(v.real()), im = split(v.imag());
        ia[(size_t)k] = make_float4(re.x, re.y, im.x, im.y);
      }
      if ((e = upload(&pl->ffc_rows, rows, &bytes))) return fail("compact factors", e);
      if ((e = upload(&pl->ffc_ia, ia, &bytes))) return fail("compact factors", e);
    }
    const size_t nfac = (size_t)fac_ncomp(*pl) * pl->nrows * P;
    if ((e = dalloc(&pl->fac_fwd, nfac, &bytes))) return fail("factors", e);
    if ((e = launch_factor_setup(*pl, false, 0))) return fail("factor setup", e);
    if (pl->ff) {
      const rexi_status r = take_range_error(*pl, "plan: float-float factors");
      if (r != REXI_OK) return r;
    }
  }

  // ---- grid, Legendre tables, FFT
  {  // tables serve the grid layout and rexi_analyze / rexi_synthesize
    std::vector<double> mu, w;
    gauss_legendre_host(pl->nlat, mu, w);
    if ((e = upload(&pl->mu_dev, mu, &bytes))) return fail("mu", e);
    const int J = pl->J, nlat = pl->nlat;
    if ((e = dalloc(&pl->tabP, (size_t)NS * J, &bytes))) return fail("tables", e);
    if ((e = dalloc(&pl->tabH, (size_t)NS * J, &bytes))) return fail("tables", e);
    {
      const int64_t cols = (int64_t)(N + 1) * J;
      alp_tables_kernel<<<(unsigned)((cols + 127) / 128), 128>>>(pl->mu_dev, N, J, pl->tabP, pl->tabH);
      if ((e = cudaGetLastError())) return fail("tables", e);
    }
    std::vector<double> sin_(3 * nlat), sout(3 * nlat);
    for (int j = 0; j < nlat; ++j) {
      const double cl = std::sqrt(1.0 - mu[j] * mu[j]);
      sin_[0 * nlat + j] = prm.gravity * w[j];
      sin_[1 * nlat + j] = cl * w[j] / (a * (1.0 - mu[j] * mu[j]));
      sin_[2 * nlat + j] = sin_[1 * nlat + j];
      sout[0 * nlat + j] = 1.0 / prm.gravity;
      sout[1 * nlat + j] = 1.0 / cl;
      sout[2 * nlat + j] = 1.0 / cl;
    }
    if ((e = upload(&pl->scale_ana_in, sin_, &bytes))) return fail("scales", e);
    if ((e = upload(&pl->scale_syn_out, sout, &bytes))) return fail("scales", e);
    std::vector<double> mf(N + 1), mc(N + 1), ma(N + 1), m1(N + 1, 1.0);
    for (int m = 0; m <= N; ++m) {
      mf[m] = 1.0 / pl->nlon;
      mc[m] = m == 0 ? 1.0 : 2.0;
      ma[m] = m == 0 ? 1.0 / pl->nlon : 0.5 / pl->nlon;
    }
    if ((e = upload(&pl->mscale_fwd, mf, &bytes))) return fail("mscale", e);
    if ((e = upload(&pl->mscale_c, mc, &bytes))) return fail("mscale", e);
    if ((e = upload(&pl->mscale_adj, ma, &bytes))) return fail("mscale", e);
    if ((e = upload(&pl->mscale_one, m1, &bytes))) return fail("mscale", e);
    {
      // binary32 copies (round to nearest even; every scale is a normal binary32 number)
      auto up32 = [&](float **d, const std::vector<double> &v) {
        std::vector<float> f(v.begin(), v.end());
        cudaError_t r = cudaMalloc(d, f.size() * sizeof(float));
        if (r == cudaSuccess) r = cudaMemcpy(*d, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
        bytes += f.size() * sizeof(float);
        return r;
      };
      if ((e = up32(&pl->scale_ana_in32, sin_)) || (e = up32(&pl->scale_syn_out32, sout)) ||
          (e = up32(&pl->mscale_fwd32, mf)) || (e = up32(&pl->mscale_c32, mc)) || (e = up32(&pl->mscale_adj32, ma)) ||
          (e = up32(&pl->mscale_one32, m1)))
        return fail("scales", e);
    }
    FftPlan &f = pl->fft;
    f.n = pl->nlon;
    fft_factor(f.n / 2, f.radix, &f.nstages);  // half-length complex FFT per real row
    f.nsplit = std::max(1, 4096 / f.n);
    std::vector<double2> tw(f.n);
    for (int k = 0; k < f.n; ++k) {
      const double th = 2.0 * M_PI * k / f.n;
      tw[k] = make_double2(std::cos(th), -std::sin(th));
    }
    double2 *twd = nullptr;
    if ((e = upload(&twd, tw, &bytes))) return fail("twiddles", e);
    f.tw_dev = twd;
    std::vector<float2> tw32(f.n);
    for (int k = 0; k < f.n; ++k) tw32[k] = make_float2((float)tw[k].x, (float)tw[k].y);
    float2 *tw32d = nullptr;
    if ((e = upload(&tw32d, tw32, &bytes))) return fail("twiddles", e);
    f.tw32_dev = tw32d;
    if ((e = fft_configure(*pl))) return fail("fft configure", e);
    if ((e = legendre_configure())) return fail("legendre configure", e);
  }

  if (prm.precision == REXI_MIXED) {
    if ((e = tc_setup(*pl))) return fail("tensor-core tables", e);
  }

  // ---- workspaces
  const int B = prm.max_batch;
  if ((e = dalloc(&pl->four, (size_t)pl->nlat * (N + 1) * 3 * B, &bytes))) return fail("fourier", e);
  if ((e = dalloc(&pl->s_in, (size_t)3 * NS * B, &bytes))) return fail("spectral", e);
  if ((e = dalloc(&pl->s_out, (size_t)3 * NS * B, &bytes))) return fail("spectral", e);
  if (pl->ff && (e = dalloc(&pl->s_ff, (size_t)3 * NS * B, &bytes))) return fail("spectral", e);
  // partial sums: at most 1024 slots and ~4 GiB (small batches need many slots to spread
  // the poles over enough warps; the reduction reads every slot once per step)
  size_t per_slot = (size_t)3 * NS * B * sizeof(double2);
  int cap = (int)std::min<size_t>(1024, std::max<size_t>(1, (size_t)(4ull << 30) / per_slot));
  cap = std::min(cap, P);
  pl->partial_cap = (size_t)cap;
  if ((e = dalloc(&pl->partial, (size_t)cap * 3 * NS * B, &bytes))) return fail("partials", e);
  pl->resident_warps = pl->num_sms * 16;
  // forward-sweep intermediates: sweep_width poles per lane per row
  if ((e = dalloc(&pl->yscratch, (size_t)pl->resident_warps * pl->lmax * sweep_width(pl->ff) * 32, &bytes)))
    return fail("scratch", e);
  if ((e = dalloc(&pl->counter, 1, &bytes))) return fail("counter", e);
  pl->slots_override = prm.pole_slots;
  if ((e = cudaDeviceSynchronize())) return fail("setup", e);
  return REXI_OK;
}

// Work list for batch B with a given number of pole groups (0: heuristic):
// items (m, slot group, first state), longest first.
// shape 0: every zonal order gets the same number of pole groups (items of different
// sizes, packed longest first); shape 1: groups in proportion to the system length
// (items of similar size, fewer partial sums for the short high orders).  Which is
// faster depends on the batch: the autotuner times both.
rexi_status build_layout(Plan &pl, int B, bool single, int groups_req, SolveLayout &L, int shape) {
  L = SolveLayout{};
  L.batch = B;
  L.shape = single ? 0 : shape;
  int bw = 1;
  while (bw < B && bw < 16) bw *= 2;
  L.bw = bw;
  const int slots_cap = (int)pl.partial_cap;
  // lanes kk >= L.kk stay idle, so slots = groups * kk never exceeds the partial buffer
  L.kk = single ? 1 : std::min(32 / (2 * bw), slots_cap);
  if (single) {
    L.groups = 1;
  } else if (groups_req > 0) {
    L.groups = std::max(1, std::min(groups_req, slots_cap / L.kk));
  } else {
    // enough items that the longest fits ~1/2 of a warp's fair share of the work
    const int nb = (B + bw - 1) / bw;
    double total = 0;
    int lmax = 0;
    for (int m = 0; m <= pl.N; ++m) {
      int l = std::max(pl.sys[2 * m].len, pl.sys[2 * m + 1].len);
      total += (double)l * pl.P * nb;
      lmax = std::max(lmax, l);
    }
    total /= L.kk;  // work per warp-lane set
    double share = total / (2.0 * pl.resident_warps);
    int g = 1;
    while (g * L.kk < slots_cap && (double)lmax * pl.P / (g * L.kk) > share) g *= 2;
    L.groups = std::max(1, std::min(g, slots_cap / L.kk));
  }
  L.slots = L.groups * L.kk;
  // pole groups per zonal order (shape 1: in proportion to its system length, the
  // longest orders getting L.groups, so that every item carries about the same work)
  int lmax = 1;
  for (int m = 0; m <= pl.N; ++m) lmax = std::max(lmax, std::max(pl.sys[2 * m].len, pl.sys[2 * m + 1].len));
  L.groups_m.assign(pl.N + 1, 1);
  std::vector<int32_t> slots_m(pl.N + 1, L.kk);
  for (int m = 0; m <= pl.N; ++m) {
    const int l = std::max(pl.sys[2 * m].len, pl.sys[2 * m + 1].len);
    L.groups_m[m] = L.shape == 0 ? L.groups
                                 : std::max(1, std::min(L.groups, (int)(((int64_t)L.groups * l + lmax - 1) / lmax)));
    slots_m[m] = L.groups_m[m] * L.kk;
  }
  struct Keyed { WorkItem w; double work; };
  std::vector<Keyed> keyed;
  const int nb = (B + bw - 1) / bw;
  for (int m = 0; m <= pl.N; ++m) {
    const int l = std::max(pl.sys[2 * m].len, pl.sys[2 * m + 1].len);
    if (l == 0) continue;
    const double work = (double)l * ((pl.P + slots_m[m] - 1) / slots_m[m]);
    for (int g = 0; g < L.groups_m[m]; ++g)
      for (int bb = 0; bb < nb; ++bb) keyed.push_back(Keyed{WorkItem{m, g, bb * bw, l}, work});
  }
  std::stable_sort(keyed.begin(), keyed.end(), [](const Keyed &x, const Keyed &y) { return x.work > y.work; });
  std::vector<WorkItem> items;
  for (const Keyed &k : keyed) items.push_back(k.w);
  L.nitems = (int)items.size();
  const size_t item_bytes = std::max<size_t>(1, items.size()) * sizeof(WorkItem);
  void *mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, item_bytes + slots_m.size() * sizeof(int32_t));
  if (e != cudaSuccess) {
    set_error(std::string("work list: ") + cudaGetErrorString(e));
    return REXI_ENOMEM;
  }
  L.items_dev = static_cast<WorkItem *>(mem);
  L.slots_m_dev = reinterpret_cast<int32_t *>(static_cast<char *>(mem) + item_bytes);
  e = cudaMemcpy(L.items_dev, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(L.slots_m_dev, slots_m.data(), slots_m.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(mem);
    L.items_dev = nullptr;
    L.slots_m_dev = nullptr;
    set_error(std::string("work list: ") + cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  return REXI_OK;
}

rexi_status get_layout(Plan &pl, int B, bool single, SolveLayout **out) {
  const int key = single ? -B : B;
  auto it = pl.layouts.find(key);
  if (it != pl.layouts.end()) {
    *out = &it->second;
    return REXI_OK;
  }
  SolveLayout L;
  // default shape: proportional groups for one or two states per warp, where the
  // uniform layout leaves most pole groups short of work
  int bw = 1;
  while (bw < B && bw < 16) bw *= 2;
  rexi_status r = build_layout(pl, B, single, single ? 1 : pl.slots_override, L, bw <= 2 ? 1 : 0);
  if (r != REXI_OK) return r;
  auto res = pl.layouts.emplace(key, L);
  *out = &res.first->second;
  return REXI_OK;
}

// Largest batch for which the untuned default is the fused solve.  Measured on GB300
// (T63-T341, M = 128-256), with each tile's poles split over the default number of CTAs:
// up to four states the fused solve is 1.03-3.4x faster than the best slot layout with
// its reduction (a single state's slot layout needs hundreds of partial sums); at eight
// states its default tile of eight is slower than the slot solve at T341.  rexi_tune
// decides per batch (and finds fused layouts that win up to sixteen states at T127-T170).
constexpr int kFusedDefaultMaxBatch = 4;

// The fused solve's layout for steps of B states, or null when the slot-partial path
// serves them: float-float solves, the Phi-only solver, the f-sphere, an explicit
// pole_slots at plan creation, a slot layout chosen for this batch (rexi_tune,
// rexi_set_pole_slots) or, without a choice, a batch above kFusedDefaultMaxBatch, or
// running sums too large for shared memory.
const FusedLayout *fused_layout(Plan &pl, int B) {
  if (pl.ff || pl.prm.solver != REXI_SOLVER_DELTA || pl.prm.fsphere) return nullptr;
  auto us = pl.use_slots.find(B);
  if (us != pl.use_slots.end() ? us->second : (pl.slots_override > 0 || B > kFusedDefaultMaxBatch)) return nullptr;
  auto it = pl.fused.find(B);
  if (it == pl.fused.end()) {
    FusedLayout F;
    auto ft = pl.fused_tile.find(B);
    auto ff = pl.fused_form.find(B);
    auto fg = pl.fused_groups.find(B);
    if (!build_fused_layout(pl, B, ft != pl.fused_tile.end() ? ft->second : 0,
                            ff != pl.fused_form.end() ? ff->second : 0, fg != pl.fused_groups.end() ? fg->second : 0, F))
      F = FusedLayout{};
    it = pl.fused.emplace(B, F).first;  // st == 0: not available
  }
  return it->second.st > 0 ? &it->second : nullptr;
}

// the fused layout for batch B with a requested CTA tile and number of pole groups (0:
// the defaults) and form (0: register; lean with CTAs of 1: four, 2: two warps),
// replacing any earlier one
const FusedLayout *set_fused_tile(Plan &pl, int B, int tile, int form = 0, int groups = 0) {
  auto it = pl.fused.find(B);
  if (it != pl.fused.end()) {
    free_fused_layout(it->second);
    pl.fused.erase(it);
  }
  pl.fused_tile[B] = tile;
  pl.fused_form[B] = form;
  pl.fused_groups[B] = groups;
  return fused_layout(pl, B);
}

// A given slot count for batch B: the layout with slots / kk pole groups replaces any
// earlier one for that batch.  Shapes 2, 3 and 4 select the fused solve instead (REXI_EINVAL
// where it does not apply), with slots = tile + 256 x pole groups.
rexi_status set_layout(Plan &pl, int B, int slots, int shape, int *used) {
  if (shape >= 2 && shape <= 4) {
    pl.use_slots[B] = false;
    if (!set_fused_tile(pl, B, slots % 256, shape - 2, slots / 256)) {
      pl.use_slots[B] = true;
      set_error("rexi_set_pole_slots: the fused solve (shapes 2, 3 and 4) needs binary64 solves of the delta "
                "solver on the rotating sphere, with running sums that fit in shared memory");
      return REXI_EINVAL;
    }
    const FusedLayout *F = fused_layout(pl, B);
    if (used) *used = F->st + 256 * F->ng;
    return REXI_OK;
  }
  SolveLayout L;
  int bw = 1;
  while (bw < B && bw < 16) bw *= 2;
  const int kk = std::max(1, std::min(32 / (2 * bw), (int)pl.partial_cap));
  rexi_status r = build_layout(pl, B, false, std::max(1, slots / kk), L, shape != 0 ? 1 : 0);
  if (r != REXI_OK) return r;
  auto it = pl.layouts.find(B);
  if (it != pl.layouts.end()) {
    cudaFree(it->second.items_dev);
    pl.layouts.erase(it);
    ++pl.layout_gen;
  }
  pl.layouts.emplace(B, L);
  pl.use_slots[B] = true;
  if (used) *used = L.slots;
  return REXI_OK;
}

// Autotuner: time the solve kernel for each candidate number of pole groups at
// batch B and keep the fastest layout for later steps with that batch.
rexi_status tune_layout(Plan &pl, int B, int *slots_out, int *shape_out) {
  cudaStream_t st = 0;
  cudaError_t e = cudaMemsetAsync(pl.s_in, 0, (size_t)3 * pl.nspec * B * sizeof(double2), st);
  if (e != cudaSuccess) {
    set_error(std::string("tune: ") + cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  SolveLayout bestL{};
  std::vector<int> tried;
  for (int cand = 0; cand < 2 * 9; ++cand) {
    const int g = 1 << (cand >> 1), shape = cand & 1;
    SolveLayout L;
    rexi_status r = build_layout(pl, B, false, g, L, shape);
    if (r != REXI_OK) {
      if (bestL.items_dev) cudaFree(bestL.items_dev);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return r;
    }
    if (std::find(tried.begin(), tried.end(), 2 * L.slots + shape) != tried.end()) {
      cudaFree(L.items_dev);
      continue;
    }
    tried.push_back(2 * L.slots + shape);
    // time the solve and the slot reduction together (more slots balance the solve
    // better but make the reduction read more partial sums)
    auto run = [&]() {
      if (pl.prm.solver == REXI_SOLVER_PHI) {
        launch_phi_solve(pl, L, pl.s_in, B, st);
        launch_phi_reduce(pl, L, pl.s_in, pl.s_out, B, st);
      } else {
        launch_solve(pl, L, false, pl.s_in, B, 0, pl.P, true, st);
        launch_reduce(pl, L, false, pl.s_in, pl.s_out, B, false, 0, st);
      }
    };
    run();  // warm-up
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 2; ++rep) run();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) {
      if (bestL.items_dev) cudaFree(bestL.items_dev);
      best = ms;
      bestL = L;
    } else {
      cudaFree(L.items_dev);
    }
  }
  // the fused solve (no slot partials, no reduction) in its CTA tiles of 32 ... 2 states,
  // with the poles of a tile split over the default number of CTAs and over 1 ... 8 CTAs
  // (up to 2 above eight states), competes with the best slot layout
  float fused_ms = 1e30f;
  int best_tile = 0, best_groups = 1;
  pl.use_slots[B] = false;
  int best_form = 0;
  for (int tile = 32; tile >= 1; tile /= 2) {
    for (int form = 0; form < 3; ++form) {
      std::vector<int> seen;
      for (int groups : {0, 1, 2, 3, 4, 6, 8}) {  // 0: the default count
        if (groups > 2 && B > 8) break;  // larger batches leave fewer schedulers idle
        const FusedLayout *F = set_fused_tile(pl, B, tile, form, groups);
        if (!F || F->st != tile) break;  // the default is smaller, or it does not fit
        if (std::find(seen.begin(), seen.end(), F->ng) != seen.end()) continue;  // capped at the passes
        seen.push_back(F->ng);
        launch_solve_fused(pl, *F, false, pl.s_in, pl.s_out, B, st);  // warm-up
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2; ++rep) launch_solve_fused(pl, *F, false, pl.s_in, pl.s_out, B, st);
        cudaEventRecord(e1, st);
        float ms = 1e30f;
        if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (ms < fused_ms) {
          fused_ms = ms;
          best_tile = tile;
          best_form = form;
          best_groups = F->ng;
        }
      }
    }
    if (tile <= 2 && tile < B) break;  // smaller tiles only re-read the factors more often
  }
  if (best_tile > 0) set_fused_tile(pl, B, best_tile, best_form, best_groups);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  auto it = pl.layouts.find(B);
  if (it != pl.layouts.end()) {
    cudaFree(it->second.items_dev);
    pl.layouts.erase(it);
    ++pl.layout_gen;
  }
  pl.layouts.emplace(B, bestL);
  // at a tie the fused solve is kept: no reduction kernel and a fraction of the slot
  // path's DRAM traffic for the same FP64 work
  const bool fused_wins = fused_ms <= best * 1.005f;
  pl.use_slots[B] = !fused_wins;
  if (slots_out) *slots_out = fused_wins ? best_tile + 256 * best_groups : bestL.slots;
  if (shape_out) *shape_out = fused_wins ? 2 + best_form : bestL.shape;
  return REXI_OK;
}

void free_plan(Plan *pl) {
  if (!pl) return;
  void *ptrs[] = {pl->coef_dev, pl->sys_dev, pl->m_of_dev, pl->fac_fwd, pl->fac_adj, pl->alpha_dev,
                  pl->beta_dev, pl->w_fwd, pl->w_adj, pl->rflags_dev, pl->mu_dev, pl->tabP, pl->tabH,
                  pl->tabP_hi, pl->tabP_lo, pl->tabH_hi, pl->tabH_lo, pl->scale_ana_in,
                  pl->scale_syn_out, pl->mscale_fwd, pl->mscale_c, pl->mscale_adj, pl->mscale_one,
                  pl->scale_ana_in32, pl->scale_syn_out32, pl->mscale_fwd32, pl->mscale_c32, pl->mscale_adj32,
                  pl->mscale_one32,
                  pl->zd_syn, pl->zd_ana_adj, pl->zd_one, pl->zd_mone, pl->fft.tw_dev, pl->fft.tw32_dev, pl->four,
                  pl->s_in, pl->s_out, pl->s_ff, pl->partial, pl->yscratch, pl->counter, pl->tc_tab_ana,
                  pl->tc_tab_syn, pl->tc_work_ana, pl->tc_work_syn, pl->dev_err, pl->phi_zc, pl->phi_q, pl->phi_abf, pl->ffc_rows, pl->ffc_ia};
  for (cudaEvent_t ev : pl->prof_ev) cudaEventDestroy(ev);
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (auto &kv : pl->layouts)
    if (kv.second.items_dev) cudaFree(kv.second.items_dev);
  for (auto &kv : pl->fused) free_fused_layout(kv.second);
  delete pl;
}

}  // namespace rexi
