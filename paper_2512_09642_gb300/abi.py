"""ctypes binding of the C ABI declared in include/sstep_cg.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
convert arguments: torch tensors become device pointers, the current torch CUDA stream
becomes the `stream` argument, status codes become exceptions. All arithmetic runs in
libsstep_cg.so. Importing this module fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsstep_cg.so")

SSTEP_MAX_S = 32
STATUS = {0: "SSTEP_OK", 1: "SSTEP_ERR_INVALID_ARG", 2: "SSTEP_ERR_CUDA", 3: "SSTEP_ERR_OOM",
          4: "SSTEP_ERR_NUMERICAL", 5: "SSTEP_ERR_NO_CONVERGENCE", 6: "SSTEP_ERR_TIMEOUT",
          7: "SSTEP_ERR_UNSUPPORTED"}
BOUNDS = {"given": 0, "gersh_lanczos10": 1, "lanczos10": 2}
GRAM_SOLVER = {"fgs": 0, "cholesky": 1}
PRECISION = {"fp64": 0, "mixed": 1}
PRECOND = {"none": 0, "jacobi": 1}
GRAM_FORM = {"direct": 0, "moments": 1, "fused": 2}
STEP_KERNEL = {"auto": 0, "tma": 1, "plain": 2}


class Opts(C.Structure):
    _fields_ = [("s", C.c_int), ("nu", C.c_int), ("lambda_min", C.c_double), ("lambda_max", C.c_double),
                ("bounds_mode", C.c_int), ("tol", C.c_double), ("max_outer", C.c_int), ("gram_solver", C.c_int),
                ("precision", C.c_int), ("precond", C.c_int), ("basis_start", C.c_int), ("gram_form", C.c_int),
                ("refresh_period", C.c_int), ("max_refresh", C.c_int), ("seed", C.c_uint64),
                ("use_graph", C.c_int), ("check_every", C.c_int), ("profile_every", C.c_int),
                ("batch_chunk", C.c_int), ("batch_ctas_per_sm", C.c_int), ("block_conjugate", C.c_int),
                ("history", C.c_int), ("step_kernel", C.c_int)]


class Info(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("refreshes", C.c_int), ("status", C.c_int), ("r0_norm", C.c_double),
                ("rel_res_recursive", C.c_double), ("rel_res_true", C.c_double),
                ("lambda_min_used", C.c_double), ("lambda_max_used", C.c_double), ("min_gii", C.c_double),
                ("delta_last", C.c_double), ("ms", C.c_float), ("kernel_launches", C.c_int),
                ("prof_ms", C.c_float * 4), ("prof_launches", C.c_int * 4), ("step_tma", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status"] = STATUS.get(self.status, str(self.status))
        d["prof_ms"] = list(self.prof_ms)
        d["prof_launches"] = list(self.prof_launches)
        return d


class SStepError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2512_09642_gb300.build` "
                          "(the s-step CG library has no fallback implementation)")
    return C.CDLL(LIB_PATH)


lib = _load()

_VP, _I64, _I, _D = C.c_void_p, C.c_int64, C.c_int, C.c_double
_SIGS = {
    "sstep_cg_default_opts": (None, [C.POINTER(Opts)]),
    "sstep_cg_create_csr": (_I, [C.POINTER(_VP), _I64, _VP, _VP, _VP, C.POINTER(Opts), _VP]),
    "sstep_cg_create_stencil": (_I, [C.POINTER(_VP), _I, _I, _I, _I, _VP, C.POINTER(Opts), _VP]),
    "sstep_cg_create_box_stencil": (_I, [C.POINTER(_VP), _I, _I, _I, _I, C.POINTER(Opts), _VP]),
    "sstep_cg_solve": (_I, [_VP, _VP, _VP, C.POINTER(Info)]),
    "sstep_cg_solve_host": (_I, [_VP, _VP, _VP, C.POINTER(Info)]),
    "sstep_cg_destroy": (_I, [_VP]),
    "sstep_cg_status_string": (C.c_char_p, [_I]),
    "sstep_cg_last_error": (C.c_char_p, [_VP]),
    "sstep_cg_apply": (_I, [_VP, _VP, _VP]),
    "sstep_cg_basis": (_I, [_VP, _VP, _VP, _I64, _I]),
    "sstep_cg_gram_solve": (_I, [_VP, _VP]),
    "sstep_cg_load_basis": (_I, [_VP, _VP, _I64]),
    "sstep_cg_get_bounds": (_I, [_VP, C.POINTER(_D), C.POINTER(_D)]),
    "sstep_cg_get_residual": (_I, [_VP, _VP]),
    "sstep_cg_lanczos": (_I, [_VP, _I, C.c_uint64, _VP, _VP, C.POINTER(_I)]),
    "sstep_cg_grad_kappa": (_I, [_VP, _VP, _VP, _VP]),
    "sstep_cg_set_tolerance": (_I, [_VP, _D, _I]),
    "sstep_convert_check": (_I, [_VP, _I, _VP, _VP, _I64, _VP]),
    "sstep_cg_batch_create": (_I, [C.POINTER(_VP), _I, _VP, _VP, C.POINTER(Opts), _VP]),
    "sstep_cg_batch_layout": (_I, [_VP, _VP, _VP, _VP]),
    "sstep_cg_batch_solve": (_I, [_VP, _VP, _VP, _VP, C.POINTER(Info)]),
    "sstep_cg_batch_destroy": (_I, [_VP]),
    "sstep_cg_batch_last_error": (C.c_char_p, [_VP]),
    "sstep_coarse_fgs": (_I, [_VP, _I, _I, _I, _VP, _VP, _I, _I]),
    "sstep_gram_fgs_noalloc": (_I, [_I64, _I, _I, _I, _VP, _I64, _VP, _D, _D, _D, _VP, _VP]),
    "sstep_cg_history": (_I, [_VP, C.POINTER(C.c_double), _I, C.POINTER(C.c_int)]),
    "sstep_selftest_tma_timeout": (_I, [C.POINTER(C.c_int)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(status: int, handle=None, allow=()):
    if status != 0 and status not in allow:
        msg = lib.sstep_cg_last_error(handle)
        raise SStepError(status, msg.decode() if msg else "")
    return status


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None):
    """cudaStream_t for the call: an int is taken as a raw handle (0 = default stream),
    None means torch's current stream, else a torch.cuda.Stream."""
    if isinstance(stream, int):
        return stream or None
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def sstep_cg_default_opts(**overrides) -> Opts:
    o = Opts()
    lib.sstep_cg_default_opts(C.byref(o))
    for k, v in overrides.items():
        if k == "bounds_mode" and isinstance(v, str):
            v = BOUNDS[v]
        elif k == "gram_solver" and isinstance(v, str):
            v = GRAM_SOLVER[v]
        elif k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        elif k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        elif k == "gram_form" and isinstance(v, str):
            v = GRAM_FORM[v]
        elif k == "step_kernel" and isinstance(v, str):
            v = STEP_KERNEL[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def sstep_cg_create_csr(n: int, rowptr, colind, vals, opts: Opts, stream=None):
    h = _VP()
    st = lib.sstep_cg_create_csr(C.byref(h), int(n), _ptr(rowptr), _ptr(colind), _ptr(vals), C.byref(opts),
                                 _stream(stream))
    _check(st, None)
    return h


def sstep_cg_create_stencil(dim: int, nx: int, ny: int, nz: int, kappa, opts: Opts, stream=None):
    h = _VP()
    st = lib.sstep_cg_create_stencil(C.byref(h), int(dim), int(nx), int(ny), int(nz), _ptr(kappa), C.byref(opts),
                                     _stream(stream))
    _check(st, None)
    return h


def sstep_cg_create_box_stencil(dim: int, nx: int, ny: int, nz: int, opts: Opts, stream=None):
    h = _VP()
    st = lib.sstep_cg_create_box_stencil(C.byref(h), int(dim), int(nx), int(ny), int(nz), C.byref(opts),
                                         _stream(stream))
    _check(st, None)
    return h


COARSE_MODE = {"formed": 0, "streaming": 1}


def sstep_coarse_fgs(h, block, g, y, nu: int, mode: str = "streaming"):
    """nu coarse-grid FGS sweeps on A_c y = g (y updated in place), A_c = P^T A P for box
    aggregates of size `block` = (bx, by[, bz])."""
    bx, by, bz = (tuple(int(v) for v in block) + (1, 1))[:3]
    _check(lib.sstep_coarse_fgs(h, bx, by, bz, _ptr(g), _ptr(y), int(nu), COARSE_MODE[mode]), h)


def sstep_cg_solve(h, b, x, allow=(5,)) -> Info:
    info = Info()
    _check(lib.sstep_cg_solve(h, _ptr(b), _ptr(x), C.byref(info)), h, allow)
    return info


def sstep_cg_solve_host(h, b_np, x_np, allow=(5,)) -> Info:
    import numpy as np
    assert b_np.dtype == np.float64 and x_np.dtype == np.float64
    assert b_np.flags.c_contiguous and x_np.flags.c_contiguous
    info = Info()
    _check(lib.sstep_cg_solve_host(h, b_np.ctypes.data, x_np.ctypes.data, C.byref(info)), h, allow)
    return info


def sstep_cg_destroy(h):
    return _check(lib.sstep_cg_destroy(h))


def sstep_cg_status_string(status: int) -> str:
    return lib.sstep_cg_status_string(int(status)).decode()


def sstep_cg_last_error(h=None) -> str:
    return lib.sstep_cg_last_error(h).decode()


def sstep_cg_apply(h, x, y):
    return _check(lib.sstep_cg_apply(h, _ptr(x), _ptr(y)), h)


def sstep_cg_basis(h, r, P, ldp: int, ncols: int):
    return _check(lib.sstep_cg_basis(h, _ptr(r), _ptr(P), int(ldp), int(ncols)), h)


def sstep_cg_load_basis(h, P, ldp: int):
    return _check(lib.sstep_cg_load_basis(h, _ptr(P), int(ldp)), h)


def sstep_cg_gram_solve(h, s: int):
    """Returns (alpha, d, c~, G~) as numpy arrays."""
    import numpy as np
    out = np.zeros(3 * s + s * s)
    _check(lib.sstep_cg_gram_solve(h, out.ctypes.data), h)
    return out[:s].copy(), out[s:2 * s].copy(), out[2 * s:3 * s].copy(), out[3 * s:].reshape(s, s).copy()


def sstep_cg_get_bounds(h):
    lo, hi = _D(), _D()
    _check(lib.sstep_cg_get_bounds(h, C.byref(lo), C.byref(hi)), h)
    return lo.value, hi.value


def sstep_cg_get_residual(h, r):
    return _check(lib.sstep_cg_get_residual(h, _ptr(r)), h)


def sstep_cg_lanczos(h, k: int, seed: int):
    import numpy as np
    a = np.zeros(k)
    b = np.zeros(max(k - 1, 1))
    steps = _I()
    _check(lib.sstep_cg_lanczos(h, int(k), int(seed), a.ctypes.data, b.ctypes.data, C.byref(steps)), h)
    m = steps.value
    return a[:m].copy(), b[:max(m - 1, 0)].copy()


def sstep_cg_grad_kappa(h, x, lam, g):
    return _check(lib.sstep_cg_grad_kappa(h, _ptr(x), _ptr(lam), _ptr(g)), h)


def sstep_cg_set_tolerance(h, tol: float, max_outer: int):
    return _check(lib.sstep_cg_set_tolerance(h, float(tol), int(max_outer)), h)


def sstep_convert_check(x, k: int, out, back, stream=None):
    return _check(lib.sstep_convert_check(_ptr(x), int(k), _ptr(out), _ptr(back), x.numel(), _stream(stream)))


def _bcheck(status, h, allow=()):
    if status != 0 and status not in allow:
        msg = lib.sstep_cg_batch_last_error(h)
        raise SStepError(status, msg.decode() if msg else "")
    return status


def sstep_cg_batch_create(grids, kappas, opts: Opts, stream=None):
    """grids: list of (nx, ny[, nz]); kappas: list of CUDA tensors or None (Poisson)."""
    import numpy as np
    g = np.zeros((len(grids), 4), dtype=np.int32)
    for i, d in enumerate(grids):
        d = tuple(int(v) for v in d)
        g[i] = (len(d),) + (d + (1, 1))[:3]
    kp = (_VP * len(grids))(*[(_ptr(k) if k is not None else None) for k in kappas])
    h = _VP()
    st = lib.sstep_cg_batch_create(C.byref(h), len(grids), g.ctypes.data, kp, C.byref(opts), _stream(stream))
    _bcheck(st, None)
    return h


def sstep_cg_batch_layout(h, count: int):
    import numpy as np
    offs = np.zeros(count, dtype=np.int64)
    lam = np.zeros(2 * count)
    total = C.c_int64()
    _bcheck(lib.sstep_cg_batch_layout(h, offs.ctypes.data, C.byref(total), lam.ctypes.data), h)
    return offs, total.value, lam.reshape(count, 2)


def sstep_cg_batch_solve(h, b, x, count: int, allow=(5,)):
    infos = (Info * count)()
    summary = Info()
    _bcheck(lib.sstep_cg_batch_solve(h, _ptr(b), _ptr(x), infos, C.byref(summary)), h, allow)
    return [i.as_dict() for i in infos], summary.as_dict()


def sstep_cg_batch_destroy(h):
    return _bcheck(lib.sstep_cg_batch_destroy(h), None)


def sstep_cg_batch_last_error(h=None) -> str:
    return lib.sstep_cg_batch_last_error(h).decode()


def sstep_gram_fgs_noalloc(n, s, nu, gram_solver, P, ldp, mdiag, mconst, lambda_min, lambda_max, out,
                           stream=None):
    """Allocation-free Gram + FGS (see the header); out: CUDA double tensor of 3s + s*s + 1."""
    if isinstance(gram_solver, str):
        gram_solver = GRAM_SOLVER[gram_solver]
    st = lib.sstep_gram_fgs_noalloc(int(n), int(s), int(nu), int(gram_solver), _ptr(P), int(ldp), _ptr(mdiag),
                                    float(mconst), float(lambda_min), float(lambda_max), _ptr(out), _stream(stream))
    return _check(st, None)


def sstep_cg_history(h, capacity: int):
    """The last solve's per-outer-iteration records (opts.history > 0): a list of dicts with
    outer, rel_res_sq (||r_(k-1)||^2 / ||r_0||^2), delta (the Gram solve's inexactness) and
    min_gii, oldest first."""
    buf = (C.c_double * (4 * capacity))()
    cnt = C.c_int(0)
    _check(lib.sstep_cg_history(h, buf, int(capacity), C.byref(cnt)), h)
    return [{"outer": int(buf[4 * k]), "rel_res_sq": buf[4 * k + 1], "delta": buf[4 * k + 2],
             "min_gii": buf[4 * k + 3]} for k in range(cnt.value)]


def exported_names():
    return sorted(_SIGS)


def sstep_selftest_tma_timeout() -> int:
    """Runs the TMA step's bounded-wait self-test; returns the control block's state after it
    (4 = timed out, the designed outcome)."""
    st = C.c_int(-1)
    _check(lib.sstep_selftest_tma_timeout(C.byref(st)), None)
    return st.value
