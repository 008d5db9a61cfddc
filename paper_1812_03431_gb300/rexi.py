"""Python binding of librexi (include/rexi.h).

Argument marshalling only: every stage of the step runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  The library must be
built in-tree (``python -m paper_1812_03431_gb300.build`` or
``__graft_entry__.build()``); loading fails loudly if it is missing.
"""
import ctypes
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librexi.so")

REXI_OK, REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA, REXI_ERANGE, REXI_ETIMEOUT = 0, -1, -2, -3, -4, -5
REXI_FP64, REXI_MIXED = 0, 1
REXI_GRID, REXI_SPECTRAL = 0, 1
STATUS = {0: "REXI_OK", -1: "REXI_EINVAL", -2: "REXI_ENOMEM", -3: "REXI_ECUDA", -4: "REXI_ERANGE",
          -5: "REXI_ETIMEOUT"}


class rexi_params(ctypes.Structure):
    _fields_ = [
        ("ntrunc", ctypes.c_int32), ("nlat", ctypes.c_int32), ("nlon", ctypes.c_int32),
        ("M", ctypes.c_int32), ("h", ctypes.c_double), ("tau", ctypes.c_double),
        ("radius", ctypes.c_double), ("omega", ctypes.c_double), ("gravity", ctypes.c_double),
        ("mean_depth", ctypes.c_double), ("normalize", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("layout", ctypes.c_int32), ("max_batch", ctypes.c_int32),
        ("strict_range", ctypes.c_int32), ("pole_slots", ctypes.c_int32),
        ("alpha", ctypes.POINTER(ctypes.c_double)), ("beta", ctypes.POINTER(ctypes.c_double)),
        ("npoles", ctypes.c_int32), ("fsphere", ctypes.c_int32), ("solver", ctypes.c_int32),
        ("solve_arith", ctypes.c_int32), ("pole_begin", ctypes.c_int32), ("pole_end", ctypes.c_int32),
    ]


class RexiError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s failed: %s (%s)" % (fn, STATUS.get(status, status), msg))
        self.status = status


_lib = None
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "rexi_params_default": (None, [ctypes.POINTER(rexi_params)]),
    "rexi_params_size": (ctypes.c_size_t, []),
    "rexi_integrate": (_I32, [_VP, _VP, _VP, _I32, _I32, _VP]),
    "rexi_set_pole_slots": (ctypes.c_int32, [_VP, _I32, _I32, _I32, ctypes.POINTER(_I32)]),
    "rexi_coefficients": (_I32, [_I32, ctypes.c_double, _I32, _DP, _DP, ctypes.POINTER(_I32), _DP]),
    "rexi_plan_create": (_I32, [ctypes.POINTER(rexi_params), ctypes.POINTER(_VP)]),
    "rexi_step": (_I32, [_VP, _VP, _VP, _I32, _VP]),
    "rexi_step_adjoint": (_I32, [_VP, _VP, _VP, _I32, _VP]),
    "rexi_step_static": (_I32, [_VP, _VP, _VP, _I32, _VP]),
    "rexi_analyze": (_I32, [_VP, _VP, _VP, _I32, _VP]),
    "rexi_synthesize": (_I32, [_VP, _VP, _VP, _I32, _VP]),
    "rexi_solve_pole": (_I32, [_VP, _I32, _VP, _VP, _I32, _VP]),
    "rexi_get_coefficients": (_I32, [_VP, _DP, _DP, ctypes.POINTER(_I32)]),
    "rexi_plan_info": (_I32, [_VP, ctypes.POINTER(ctypes.c_int64), _I32]),
    "rexi_tune": (_I32, [_VP, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "rexi_ragged_create": (_I32, [ctypes.POINTER(_VP), _I32, _I32, ctypes.POINTER(_VP)]),
    "rexi_ragged_step": (_I32, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_I32), _I32, _VP]),
    "rexi_ragged_destroy": (None, [_VP]),
    "rexi_profile_enable": (_I32, [_VP, _I32]),
    "rexi_profile_read": (_I32, [_VP, _DP, _I32, ctypes.POINTER(_I32)]),
    "rexi_check_device": (_I32, [_VP]),
    "rexi_destroy": (None, [_VP]),
    "rexi_last_error": (ctypes.c_char_p, []),
    "rexi_measure_fp64_fma": (_I32, [_I32, _DP, _DP, _VP]),
    "rexi_inject_device_error": (_I32, [_VP, _I32]),
}


def load():
    """Load librexi.so from the package directory (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librexi.so not found at %s: build it first "
                               "(python -m paper_1812_03431_gb300.build)" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if lib.rexi_params_size() != ctypes.sizeof(rexi_params):
            raise RuntimeError("rexi_params: the binding's struct (%d bytes) does not match the library's (%d)"
                               % (ctypes.sizeof(rexi_params), lib.rexi_params_size()))
        _lib = lib
    return _lib


def _read_json(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _check(fn, status):
    if status != REXI_OK:
        raise RexiError(fn, status, load().rexi_last_error().decode())


# ---- same-named thin wrappers --------------------------------------------------------
def rexi_params_default():
    p = rexi_params()
    load().rexi_params_default(ctypes.byref(p))
    return p


def rexi_coefficients(M, h, normalize=True):
    """Host-side T-REXI poles: returns (alpha, beta, eps) as complex128 arrays and float."""
    P = 2 * (M + 11) + 1
    al = np.zeros(2 * P)
    be = np.zeros(2 * P)
    n = _I32()
    eps = ctypes.c_double()
    _check("rexi_coefficients", load().rexi_coefficients(
        M, h, int(normalize), al.ctypes.data_as(_DP), be.ctypes.data_as(_DP), ctypes.byref(n),
        ctypes.byref(eps)))
    return al.view(np.complex128)[: n.value].copy(), be.view(np.complex128)[: n.value].copy(), eps.value


def rexi_measure_fp64_fma(reps=5, stream=None):
    """Measured binary64 FMA rate of the current device (TFLOP/s, best of ``reps``
    launches) and that launch's milliseconds (include/rexi_measure.h)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check("rexi_measure_fp64_fma", load().rexi_measure_fp64_fma(int(reps), ctypes.byref(tf), ctypes.byref(ms),
                                                                  _stream_handle(stream)))
    return tf.value, ms.value


def pole_shard(P, rank, world):
    """Rank `rank`'s contiguous share [begin, end) of P poles split evenly over `world`
    ranks (sizes differ by at most one; the first P mod world ranks take one more), the
    even split of the REXI terms over ranks of Sec. 6.4."""
    if not (0 <= rank < world) or P < world:
        raise ValueError("need 0 <= rank < world <= P")
    q, r = divmod(P, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A librexi plan: one T-REXI step of the linear SWE for a fixed truncation, grid and poles.

    ``precision`` selects the transforms ("fp64", or "mixed": 3xTF32 Legendre and FP32
    FFTs); ``solve_arith`` the arithmetic of the banded solves and the pole sum ("fp64",
    or "fp32x2": float-float pairs of FP32 on the FP32 pipes, 48-bit significands)."""

    def __init__(self, N, nlat=None, nlon=None, M=128, h=0.2, tau=3600.0, max_batch=1,
                 layout="grid", precision="fp64", normalize=True, alpha=None, beta=None,
                 radius=6.37122e6, omega=7.292e-5, gravity=9.80616, mean_depth=1.0e4,
                 pole_slots=0, strict_range=False, fsphere=False, solver="delta", solve_arith="fp64",
                 poles=None):
        lib = load()
        p = rexi_params()
        lib.rexi_params_default(ctypes.byref(p))
        if nlon is None:
            nlon = 3 * N + 3
            while any(nlon % q == 0 for q in ()) or not _smooth(nlon):
                nlon += 1
            nlon += nlon % 2
        if nlat is None:
            nlat = nlon // 2
        p.ntrunc, p.nlat, p.nlon, p.M, p.h, p.tau = N, nlat, nlon, M, h, tau
        p.radius, p.omega, p.gravity, p.mean_depth = radius, omega, gravity, mean_depth
        p.normalize = int(normalize)
        p.precision = {"fp64": REXI_FP64, "mixed": REXI_MIXED}[precision]
        p.layout = {"grid": REXI_GRID, "spectral": REXI_SPECTRAL}[layout]
        p.max_batch = max_batch
        p.strict_range = int(strict_range)
        p.pole_slots = pole_slots
        p.fsphere = 1 if fsphere else 0
        p.solver = {"delta": 0, "phi": 1}[solver]
        p.solve_arith = {"fp64": 0, "fp32x2": 1}[solve_arith]
        if poles is not None:  # (begin, end): this plan's share of the poles (pole_shard)
            p.pole_begin, p.pole_end = int(poles[0]), int(poles[1])
        self._keep = []
        if alpha is not None:
            al = np.ascontiguousarray(np.asarray(alpha, dtype=np.complex128)).view(np.float64)
            be = np.ascontiguousarray(np.asarray(beta, dtype=np.complex128)).view(np.float64)
            self._keep = [al, be]
            p.alpha = al.ctypes.data_as(_DP)
            p.beta = be.ctypes.data_as(_DP)
            p.npoles = al.size // 2
        h_ = _VP()
        _check("rexi_plan_create", lib.rexi_plan_create(ctypes.byref(p), ctypes.byref(h_)))
        self._h = h_
        self.N, self.nlat, self.nlon, self.max_batch = N, nlat, nlon, max_batch
        self.layout, self.precision, self.solver = layout, precision, solver
        self.solve_arith = solve_arith
        self.layout_shape = {}
        self.nspec = (N + 1) * (N + 2) // 2

    # -- helpers
    def _io(self, x, out, grid):
        import torch
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("input must be a contiguous CUDA tensor")
        if grid:
            if x.dtype != torch.float64 or tuple(x.shape[1:]) != (3, self.nlat, self.nlon):
                raise ValueError("grid input must be float64 [B, 3, nlat, nlon]")
            shape, dt = x.shape, torch.float64
        else:
            if x.dtype != torch.complex128 or tuple(x.shape[1:]) != (3, self.nspec):
                raise ValueError("spectral input must be complex128 [B, 3, nspec]")
            shape, dt = x.shape, torch.complex128
        if out is None:
            out = torch.empty(shape, dtype=dt, device=x.device)
        return out

    def step(self, x, out=None, stream=None):
        out = self._io(x, out, self.layout == "grid")
        _check("rexi_step", load().rexi_step(self._h, x.data_ptr(), out.data_ptr(), x.shape[0],
                                              _stream_handle(stream)))
        return out

    def integrate(self, x, nsteps, out=None, stream=None):
        """rexi_integrate: nsteps consecutive steps from x in one call (the state stays in
        spectral space in between)."""
        out = self._io(x, out, self.layout == "grid")
        _check("rexi_integrate", load().rexi_integrate(self._h, x.data_ptr(), out.data_ptr(), x.shape[0],
                                                        int(nsteps), _stream_handle(stream)))
        return out

    def step_adjoint(self, g, out=None, stream=None):
        out = self._io(g, out, self.layout == "grid")
        _check("rexi_step_adjoint", load().rexi_step_adjoint(self._h, g.data_ptr(), out.data_ptr(),
                                                              g.shape[0], _stream_handle(stream)))
        return out

    def step_static(self, x, out=None, stream=None):
        """rexi_step_static: the spectral step with all per-call scratch in the library's
        fixed 64 MiB device array (allocates nothing); see include/rexi.h."""
        out = self._io(x, out, False)
        _check("rexi_step_static", load().rexi_step_static(self._h, x.data_ptr(), out.data_ptr(),
                                                            x.shape[0], _stream_handle(stream)))
        return out

    def analyze(self, grid, stream=None):
        import torch
        self._io(grid, grid, True)
        out = torch.empty((grid.shape[0], 3, self.nspec), dtype=torch.complex128, device=grid.device)
        _check("rexi_analyze", load().rexi_analyze(self._h, grid.data_ptr(), out.data_ptr(),
                                                    grid.shape[0], _stream_handle(stream)))
        return out

    def synthesize(self, spec, stream=None):
        import torch
        self._io(spec, spec, False)
        out = torch.empty((spec.shape[0], 3, self.nlat, self.nlon), dtype=torch.float64, device=spec.device)
        _check("rexi_synthesize", load().rexi_synthesize(self._h, spec.data_ptr(), out.data_ptr(),
                                                          spec.shape[0], _stream_handle(stream)))
        return out

    def solve_pole(self, k, x, out=None, stream=None):
        out = self._io(x, out, False)
        _check("rexi_solve_pole", load().rexi_solve_pole(self._h, k, x.data_ptr(), out.data_ptr(),
                                                          x.shape[0], _stream_handle(stream)))
        return out

    def coefficients(self):
        P = self.info()["P"]
        al = np.zeros(2 * P)
        be = np.zeros(2 * P)
        n = _I32()
        _check("rexi_get_coefficients", load().rexi_get_coefficients(
            self._h, al.ctypes.data_as(_DP), be.ctypes.data_as(_DP), ctypes.byref(n)))
        return al.view(np.complex128).copy(), be.view(np.complex128).copy()

    def tune(self, batch, cache=None):
        """rexi_tune: time the solve and reduction for several pole-group counts and both
        slot-layout shapes at this batch size, and the fused solve (shapes 2 to 4, no slots)
        where it applies, and keep the fastest; returns the chosen number of pole slots (for the
        fused solve its tile + 256 x its pole groups; the shape is kept in
        ``self.layout_shape[batch]``).

        ``cache``: path of a JSON file of earlier choices keyed by the plan's shape (N,
        grid, P, batch, precision, solver, solve arithmetic) and the GPU's name; a hit sets the layout
        without timing (rexi_set_pole_slots), a miss tunes and records the result."""
        key = None
        if cache:
            key = self._tune_key(batch)
            table = _read_json(cache)
            if key in table:
                slots, shape = table[key]
                return self.set_pole_slots(batch, int(slots), int(shape))
        n, sh = _I32(), _I32()
        _check("rexi_tune", load().rexi_tune(self._h, batch, ctypes.byref(n), ctypes.byref(sh)))
        self.layout_shape[batch] = sh.value
        if cache:
            table = _read_json(cache)
            table[key] = [n.value, sh.value]
            tmp = cache + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return n.value

    def set_pole_slots(self, batch, slots, shape=0, groups=0):
        """rexi_set_pole_slots: use this pole-slot count and layout shape (0: the same groups
        for every zonal order, 1: in proportion to the system length) for this batch size,
        or shape 2 (3: its lean form, 4: the lean form on two-warp CTAs): the fused solve with
        ``slots`` states per CTA tile (0: default) and each tile's poles split over ``groups``
        CTAs (0: default).  For shapes 2 to 4 returns tile + 256 x groups as used (``slots``
        may carry that packing itself, as rexi_tune returns it)."""
        n = _I32()
        if shape >= 2:
            slots = slots + 256 * groups
        _check("rexi_set_pole_slots", load().rexi_set_pole_slots(self._h, batch, slots, shape, ctypes.byref(n)))
        self.layout_shape[batch] = shape
        return n.value

    def _tune_key(self, batch):
        import torch
        i = self.info()
        gpu = torch.cuda.get_device_name(torch.cuda.current_device())
        return "N%d_%dx%d_P%d_B%d_%s_%s_%s_%s_%s" % (i["N"], i["nlon"], i["nlat"], i["P"], batch, self.precision,
                                                     self.solver, self.solve_arith, self.layout, gpu)

    def info(self):
        v = (ctypes.c_int64 * 8)()
        _check("rexi_plan_info", load().rexi_plan_info(self._h, v, 8))
        keys = ["N", "nspec", "P", "nlat", "nlon", "max_batch", "pole_slots", "device_bytes"]
        return dict(zip(keys, list(v)))

    def check_device(self):
        """Raise RexiError(REXI_ETIMEOUT) if a bounded device wait of this plan expired, or
        RexiError(REXI_ERANGE) if a float-float solve met a value beyond binary32's range."""
        _check("rexi_check_device", load().rexi_check_device(self._h))

    def inject_device_error(self, bits):
        """rexi_inject_device_error: set error bits (1 timeout, 2 range) in the plan's device
        error word from the host, for tests of check_device."""
        _check("rexi_inject_device_error", load().rexi_inject_device_error(self._h, int(bits)))

    STAGES = ["fft_fwd", "leg_ana", "solve", "reduce", "leg_syn", "fft_inv", "transpose_in", "transpose_out"]

    def profile_enable(self, max_calls):
        _check("rexi_profile_enable", load().rexi_profile_enable(self._h, max_calls))

    def profile_read(self):
        ms = np.zeros(8)
        n = _I32()
        _check("rexi_profile_read", load().rexi_profile_read(self._h, ms.ctypes.data_as(_DP), 8, ctypes.byref(n)))
        return dict(zip(self.STAGES, ms.tolist())), n.value

    def close(self):
        if getattr(self, "_h", None):
            load().rexi_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ragged:
    """Ragged batch over several REXI_SPECTRAL plans: one persistent solve launch for all states."""

    def __init__(self, plans, max_states):
        arr = (_VP * len(plans))(*[p._h for p in plans])
        h = _VP()
        _check("rexi_ragged_create", load().rexi_ragged_create(arr, len(plans), max_states, ctypes.byref(h)))
        self._h = h
        self.plans = list(plans)

    def step(self, states, outs, state_plan, stream=None):
        """states/outs: lists of complex128 CUDA tensors [3, nspec_p]; state_plan: plan index per state."""
        n = len(states)
        ins = (_VP * n)(*[t.data_ptr() for t in states])
        ous = (_VP * n)(*[t.data_ptr() for t in outs])
        sp = (_I32 * n)(*state_plan)
        _check("rexi_ragged_step", load().rexi_ragged_step(self._h, ins, ous, sp, n, _stream_handle(stream)))
        return outs

    def close(self):
        if getattr(self, "_h", None):
            load().rexi_ragged_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _smooth(n):
    for q in (2, 3, 5):
        while n % q == 0:
            n //= q
    return n == 1
