"""Numerical dispersion analysis of the T-REXI step (paper Sec. 6.3).

The propagator E (U_{n+1} = E U_n) is obtained column by column, as the paper
does: each real degree of freedom of the spectral state is activated alone and
one step is taken.  Here all columns are one batched ``rexi_step`` on the GPU.
The logarithm of E's eigenvalues gives the numerical frequencies; with a step
small enough that the logarithm stays on its principal branch (the paper uses
dt <= 400 s at T16) they are compared with the exact frequencies of L.

Real coordinates of a spectral state [3, nspec]: Re of every coefficient except
zeta_0^0 and delta_0^0 (not state), and Im of every m > 0 coefficient.
"""
import numpy as np


def real_coordinates(N):
    """List of (field, idx, part) for the real degrees of freedom (part 0 = Re, 1 = Im)."""
    coords = []
    for f in range(3):
        i = 0
        for m in range(N + 1):
            for n in range(m, N + 1):
                if not (f > 0 and m == 0 and n == 0):
                    coords.append((f, i, 0))
                    if m > 0:
                        coords.append((f, i, 1))
                i += 1
    return coords


def probe_states(N):
    """[n, 3, nspec] complex: state k is the k-th real coordinate set to one."""
    coords = real_coordinates(N)
    nspec = (N + 1) * (N + 2) // 2
    probes = np.zeros((len(coords), 3, nspec), dtype=np.complex128)
    for k, (f, i, part) in enumerate(coords):
        probes[k, f, i] = 1.0 if part == 0 else 1.0j
    return probes


def assemble(out, N):
    """Real matrix E from the stepped probe states: column k is the step of probe k."""
    coords = real_coordinates(N)
    E = np.empty((len(coords), len(coords)))
    for r, (f, i, part) in enumerate(coords):
        E[r] = out[:, f, i].real if part == 0 else out[:, f, i].imag
    return E


def propagator(plan, N):
    """E from one batched GPU step of a REXI_SPECTRAL plan of truncation N whose
    max_batch is at least ``len(real_coordinates(N))``."""
    import torch
    out = plan.step(torch.from_numpy(probe_states(N)).cuda()).cpu().numpy()
    return assemble(out, N)


def eigenvalues_by_phase(E):
    """Eigenvalues of E ordered by their argument (monotone in omega while |omega dt| < pi)."""
    lam = np.linalg.eigvals(E)
    return lam[np.argsort(np.angle(lam), kind="stable")]


def dispersion_relation(E, dt):
    """(omega, |lambda|) of the numerical modes, omega = arg(lambda) / dt, ordered by omega."""
    lam = eigenvalues_by_phase(E)
    return np.angle(lam) / dt, np.abs(lam)


def relative_phase_error(omega_num, omega_exact, floor=1e-12):
    """(omega_exact, omega_num / omega_exact - 1) over the non-stationary modes; both
    arrays are paired by sorting."""
    a = np.sort(omega_exact)
    b = np.sort(omega_num)
    keep = np.abs(a) > floor * np.abs(a).max()
    return a[keep], b[keep] / a[keep] - 1.0
