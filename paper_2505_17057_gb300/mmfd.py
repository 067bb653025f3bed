"""ctypes binding of the C ABI in include/mmfd.h (argument marshalling only).

Every computation runs inside libmmfd.so.  PyTorch is used, optionally, for
device memory (the caching allocator behind the library's allocator callback)
and streams.  Importing this module loads the library; if it has not been
built, the import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmmfd.so")

# status codes
MMFD_OK = 0
MMFD_PENDING = 1
MMFD_ERR_ARG = -1
MMFD_ERR_UNSUPPORTED = -2
MMFD_ERR_UNREPRESENTABLE = -3
MMFD_ERR_UNSTABLE = -4
MMFD_ERR_OOM = -5
MMFD_ERR_ADMISSION = -6
MMFD_ERR_NONFINITE = -7
MMFD_ERR_TIMEOUT = -8
MMFD_ERR_CUDA = -9
MMFD_ERR_STATE = -10

MMFD_LCDE, MMFD_NCDE, MMFD_NSE, MMFD_LWE = 0, 1, 2, 3
MMFD_D2Q5, MMFD_D2Q9, MMFD_D3Q7, MMFD_D3Q19 = 0, 1, 2, 3
MMFD_FP64, MMFD_FP32, MMFD_BF16 = 0, 1, 2
MMFD_HOST, MMFD_DEVICE = 0, 1
MMFD_DT_F64, MMFD_DT_F32 = 0, 1
MMFD_COEF_EXPLICIT, MMFD_COEF_TARGETS = 0, 1
MMFD_FLAG_ALLOW_UNSTABLE = 0x1
MMFD_FLAG_DROP_OFFDIAG = 0x2
MMFD_FLAG_STOCHASTIC_ROUND = 0x4
MMFD_FLAG_TWO_SETS = 0x8
MMFD_FLAG_THETA = 0x10
MMFD_BC_PERIODIC, MMFD_BC_DIRICHLET = 0, 1
MMFD_RED_SUM, MMFD_RED_MAXABS, MMFD_RED_NONFINITE = 0, 1, 2
MMFD_SRC_NONE, MMFD_SRC_S, MMFD_SRC_SU, MMFD_SRC_SM = 0, 1, 2, 3

PDE = {"LCDE": MMFD_LCDE, "NCDE": MMFD_NCDE, "NSE": MMFD_NSE, "LWE": MMFD_LWE}
LATTICE = {"D2Q5": MMFD_D2Q5, "D2Q9": MMFD_D2Q9, "D3Q7": MMFD_D3Q7, "D3Q19": MMFD_D3Q19}
STORAGE = {"fp64": MMFD_FP64, "fp32": MMFD_FP32, "bf16": MMFD_BF16}
SOURCE = {"none": MMFD_SRC_NONE, "s": MMFD_SRC_S, "su": MMFD_SRC_SU, "sm": MMFD_SRC_SM}

ALLOC_FN = C.CFUNCTYPE(C.c_int, C.c_size_t, C.POINTER(C.c_void_p), C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class mmfd_desc(C.Structure):
    _fields_ = [
        ("pde", C.c_int), ("lattice", C.c_int), ("levels", C.c_int), ("dim", C.c_int),
        ("n", C.c_longlong * 3), ("dt", C.c_double), ("dx", C.c_double * 3), ("d0", C.c_double * 3),
        ("K", (C.c_double * 3) * 3), ("u", C.c_double * 3), ("lambda_bar", C.c_double),
        ("flux", (C.c_double * 4) * 3), ("diff", C.c_double * 4), ("rho0", C.c_double),
        ("coef_mode", C.c_int),
        ("a", C.c_double * 3), ("ahat", C.c_double * 3), ("abar", C.c_double * 3), ("abarhat", C.c_double * 3),
        ("targets", C.c_double * 5), ("targets_bar", C.c_double * 5),
        ("d2", (C.c_double * 3) * 2), ("d1", (C.c_double * 3) * 2),
        ("bar_d2", (C.c_double * 3) * 2), ("bar_d1", (C.c_double * 3) * 2),
        ("storage", C.c_int), ("flags", C.c_uint), ("ref", C.c_double * 4), ("temporal_depth", C.c_int),
        ("seed", C.c_ulonglong), ("stream", C.c_void_p),
        ("alloc", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("source", C.c_int), ("b", C.c_double * 3), ("bhat", C.c_double * 3),
        ("theta", C.c_double), ("boundary", C.c_int),
    ]


class mmfd_info_t(C.Structure):
    _fields_ = [
        ("nf", C.c_int), ("levels_stored", C.c_int),
        ("a", C.c_double * 3), ("ahat", C.c_double * 3), ("abar", C.c_double * 3), ("abarhat", C.c_double * 3),
        ("A10", C.c_double), ("A20", C.c_double), ("A21", C.c_double), ("A22", C.c_double),
        ("c", C.c_double * 3), ("d0", C.c_double * 3), ("cs2", C.c_double * 3), ("w", C.c_double * 19),
        ("Cmat", (C.c_double * 3) * 3), ("m2", C.c_double * 5), ("max_lambda", C.c_double),
        ("bytes_per_lu", C.c_double), ("device_bytes", C.c_longlong), ("temporal_depth", C.c_int),
        ("steps_done", C.c_longlong), ("kernel", C.c_char * 32), ("sweeps", C.c_int), ("tile_rows", C.c_int),
    ]


class mmfd_tune_info(C.Structure):
    _fields_ = [("temporal_depth", C.c_int), ("rows_per_item", C.c_int), ("ms_per_step", C.c_double),
                ("candidates", C.c_int), ("from_cache", C.c_int)]


class mmfd_server_desc(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_slots", C.c_int), ("steps_per_tick", C.c_int),
                ("use_graphs", C.c_int), ("stream", C.c_void_p)]


class mmfd_result(C.Structure):
    _fields_ = [("status", C.c_int), ("steps_done", C.c_longlong), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("finish_s", C.c_double), ("nf", C.c_int), ("n", C.c_longlong * 3)]


class mmfd_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("admitted", C.c_longlong), ("finished", C.c_longlong),
                ("rejected", C.c_longlong), ("lattice_updates", C.c_longlong), ("ticks", C.c_longlong),
                ("launches", C.c_longlong), ("graph_replays", C.c_longlong), ("bytes_in_use", C.c_size_t),
                ("active", C.c_int)]


# every function declared in include/mmfd.h, with its ctypes signature
_VP = C.c_void_p
_PV = C.POINTER(C.c_void_p)
SIGNATURES = {
    "mmfd_desc_init": (C.c_int, [C.POINTER(mmfd_desc)]),
    "mmfd_create": (C.c_int, [C.POINTER(mmfd_desc), _PV]),
    "mmfd_set_fields": (C.c_int, [_VP, C.c_int, _PV, C.c_int, C.c_int]),
    "mmfd_set_source": (C.c_int, [_VP, C.c_int, _PV, C.c_int, C.c_int]),
    "mmfd_set_boundary": (C.c_int, [_VP, _PV, C.c_int, C.c_int]),
    "mmfd_step": (C.c_int, [_VP, C.c_longlong]),
    "mmfd_fields": (C.c_int, [_VP, C.c_int, _PV, C.c_int, C.c_int]),
    "mmfd_reduce": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_double)]),
    "mmfd_error_norms": (C.c_int, [_VP, C.c_int, _VP, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "mmfd_reduce_static": (C.c_int, [_VP, C.c_int, C.c_longlong, C.c_int, _VP, _VP]),
    "mmfd_linear_stability": (C.c_int, [C.POINTER(mmfd_desc), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mmfd_check_fields": (C.c_int, [_VP, C.POINTER(C.c_double)]),
    "mmfd_set_rows": (C.c_int, [_VP, C.c_int, C.c_longlong, C.c_longlong, _PV, C.c_int, C.c_int]),
    "mmfd_get_rows": (C.c_int, [_VP, C.c_int, C.c_longlong, C.c_longlong, _PV, C.c_int, C.c_int]),
    "mmfd_get_info": (C.c_int, [_VP, C.POINTER(mmfd_info_t)]),
    "mmfd_autotune": (C.c_int, [_VP, C.c_char_p, C.POINTER(mmfd_tune_info)]),
    "mmfd_set_stream": (C.c_int, [_VP, _VP]),
    "mmfd_destroy": (C.c_int, [_VP]),
    "mmfd_solve_three_level": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mmfd_trt_coefficients": (C.c_int, [C.c_double] + [C.POINTER(C.c_double)] * 4),
    "mmfd_wave_coefficients": (C.c_int, [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mmfd_describe": (C.c_int, [C.POINTER(mmfd_desc), C.POINTER(mmfd_info_t)]),
    "mmfd_selftest_wait_timeout": (C.c_int, [_VP, C.c_longlong]),
    "mmfd_strerror": (C.c_char_p, [C.c_int]),
    "mmfd_last_error": (C.c_char_p, []),
    "mmfd_server_create": (C.c_int, [C.POINTER(mmfd_server_desc), _PV]),
    "mmfd_submit": (C.c_int, [_VP, C.POINTER(mmfd_desc), _PV, C.c_int, C.c_longlong, C.POINTER(C.c_ulonglong)]),
    "mmfd_poll": (C.c_int, [_VP, C.c_ulonglong, C.POINTER(mmfd_result)]),
    "mmfd_server_drain": (C.c_int, [_VP]),
    "mmfd_result_fields": (C.c_int, [_VP, C.c_ulonglong, _PV, C.c_int, C.c_int]),
    "mmfd_release": (C.c_int, [_VP, C.c_ulonglong]),
    "mmfd_server_get_stats": (C.c_int, [_VP, C.POINTER(mmfd_server_stats)]),
    "mmfd_server_destroy": (C.c_int, [_VP]),
}


class MMFDError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        extra = last_error()
        if extra:
            msg += f": {extra}"
        super().__init__(msg)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2505_17057_gb300.build.build() "
                          "(the MMFD path has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def strerror(code: int) -> str:
    return lib.mmfd_strerror(int(code)).decode()


def last_error() -> str:
    return lib.mmfd_last_error().decode()


def check(rc: int, where: str) -> int:
    if rc < 0:
        raise MMFDError(rc, where)
    return rc


# ------------------------------------------------------------------ thin functions, same names

def mmfd_desc_init() -> mmfd_desc:
    d = mmfd_desc()
    check(lib.mmfd_desc_init(C.byref(d)), "mmfd_desc_init")
    return d


def mmfd_describe(d: mmfd_desc) -> mmfd_info_t:
    info = mmfd_info_t()
    check(lib.mmfd_describe(C.byref(d), C.byref(info)), "mmfd_describe")
    return info


def mmfd_solve_three_level(targets: Sequence[float]):
    t = (C.c_double * 5)(*[float(v) for v in targets])
    a = (C.c_double * 3)()
    ah = (C.c_double * 3)()
    check(lib.mmfd_solve_three_level(t, a, ah), "mmfd_solve_three_level")
    return tuple(a), tuple(ah)


def mmfd_trt_coefficients(s_minus: float) -> dict:
    """Keyword arguments a, ahat, abar, abarhat of make_desc for the TRT special case."""
    out = [(C.c_double * 3)() for _ in range(4)]
    check(lib.mmfd_trt_coefficients(float(s_minus), *out), "mmfd_trt_coefficients")
    return dict(zip(("a", "ahat", "abar", "abarhat"), (tuple(o) for o in out)))


def mmfd_wave_coefficients(gamma: float) -> dict:
    """Keyword arguments a, ahat of make_desc for the wave-equation scheme."""
    a, ah = (C.c_double * 3)(), (C.c_double * 3)()
    check(lib.mmfd_wave_coefficients(float(gamma), a, ah), "mmfd_wave_coefficients")
    return {"a": tuple(a), "ahat": tuple(ah)}


def mmfd_create(d: mmfd_desc) -> int:
    h = C.c_void_p()
    check(lib.mmfd_create(C.byref(d), C.byref(h)), "mmfd_create")
    return h.value


def _ptr_array(ptrs: Sequence[int]):
    arr = (C.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


def mmfd_set_fields(h: int, level: int, ptrs: Sequence[int], where: int, dtype: int) -> None:
    check(lib.mmfd_set_fields(h, level, _ptr_array(ptrs), where, dtype), "mmfd_set_fields")


def mmfd_set_source(h: int, level: int, ptrs: Sequence[int], where: int, dtype: int) -> None:
    check(lib.mmfd_set_source(h, level, _ptr_array(ptrs), where, dtype), "mmfd_set_source")


def mmfd_set_boundary(h: int, ptrs: Sequence[int], where: int, dtype: int) -> None:
    check(lib.mmfd_set_boundary(h, _ptr_array(ptrs), where, dtype), "mmfd_set_boundary")


def mmfd_step(h: int, nsteps: int) -> None:
    check(lib.mmfd_step(h, int(nsteps)), "mmfd_step")


def mmfd_fields(h: int, level: int, ptrs: Sequence[int], where: int, dtype: int) -> None:
    check(lib.mmfd_fields(h, level, _ptr_array(ptrs), where, dtype), "mmfd_fields")


def mmfd_reduce(h: int, what: int, nout: int) -> List[float]:
    out = (C.c_double * max(nout, 4))()
    check(lib.mmfd_reduce(h, what, out), "mmfd_reduce")
    return list(out[:nout])


def mmfd_error_norms(h: int, field: int, ref_ptr: int, where: int, dtype: int) -> List[float]:
    out = (C.c_double * 3)()
    check(lib.mmfd_error_norms(h, field, ref_ptr, where, dtype, out), "mmfd_error_norms")
    return list(out)


def mmfd_reduce_static(field_ptr: int, dtype: int, count: int, what: int, out_ptr: int,
                       stream: Optional[int]) -> None:
    check(lib.mmfd_reduce_static(field_ptr, dtype, int(count), what, out_ptr, stream), "mmfd_reduce_static")


def mmfd_linear_stability(d: mmfd_desc, state: Sequence[float]):
    """(status, max_amp): MMFD_OK or MMFD_ERR_UNSTABLE with the largest amplification modulus."""
    st = (C.c_double * 4)(*([float(v) for v in state] + [0.0] * (4 - len(state))))
    out = C.c_double(0.0)
    rc = lib.mmfd_linear_stability(C.byref(d), st, C.byref(out))
    if rc != MMFD_ERR_UNSTABLE:
        check(rc, "mmfd_linear_stability")
    return rc, out.value


def mmfd_set_rows(h: int, level: int, r0: int, count: int, ptrs: Sequence[int], where: int, dtype: int) -> None:
    check(lib.mmfd_set_rows(h, level, int(r0), int(count), _ptr_array(ptrs), where, dtype), "mmfd_set_rows")


def mmfd_get_rows(h: int, level: int, r0: int, count: int, ptrs: Sequence[int], where: int, dtype: int) -> None:
    check(lib.mmfd_get_rows(h, level, int(r0), int(count), _ptr_array(ptrs), where, dtype), "mmfd_get_rows")


def mmfd_check_fields(h: int):
    """(status, max_amp) about the current level's extreme states (MMFD_OK or MMFD_ERR_UNSTABLE)."""
    out = C.c_double(0.0)
    rc = lib.mmfd_check_fields(h, C.byref(out))
    if rc != MMFD_ERR_UNSTABLE:
        check(rc, "mmfd_check_fields")
    return rc, out.value


def mmfd_get_info(h: int) -> mmfd_info_t:
    info = mmfd_info_t()
    check(lib.mmfd_get_info(h, C.byref(info)), "mmfd_get_info")
    return info


def mmfd_autotune(h: int, cache_path: Optional[str] = None) -> mmfd_tune_info:
    info = mmfd_tune_info()
    path = cache_path.encode() if cache_path else None
    check(lib.mmfd_autotune(h, path, C.byref(info)), "mmfd_autotune")
    return info


def mmfd_selftest_wait_timeout(stream: Optional[int], budget_cycles: int) -> int:
    """Returns the status code (MMFD_ERR_TIMEOUT is the expected, passing result)."""
    return lib.mmfd_selftest_wait_timeout(stream, int(budget_cycles))


def mmfd_set_stream(h: int, stream: int) -> None:
    check(lib.mmfd_set_stream(h, stream), "mmfd_set_stream")


def mmfd_destroy(h: int) -> None:
    check(lib.mmfd_destroy(h), "mmfd_destroy")


# ------------------------------------------------------------------ descriptor helpers

def make_desc(pde: str, lattice: str, levels: int, n: Sequence[int], dt: float, dx: Sequence[float],
              storage: str = "fp32", K=None, u=None, lambda_bar: float = 1.0, flux=None, diff=None,
              rho0: float = 1.0, a=None, ahat=None, abar=None, abarhat=None, targets=None, targets_bar=None,
              d0=None, flags: int = 0, ref=None, temporal_depth: int = 1, seed: Optional[int] = None,
              stream: Optional[int] = None, sets: Optional[dict] = None, source: str = "none",
              b=None, bhat=None, theta: Optional[float] = None, boundary: str = "periodic") -> mmfd_desc:
    """Fill an mmfd_desc (plain field assignment; every derived constant is computed by the library).

    sets: the multiple-parameter-set scheme (MMFD_FLAG_TWO_SETS): a dict with "d2", "d1" and,
    for the NSE momentum, "bar_d2", "bar_d1", each a pair of triples (level t, level t - dt).
    source: "none", "s" (M_1F = 0), "su" (M_1F = S u) or "sm" (M_1F given); b, bhat: the source
    coefficient triples (None: the library's defaults).
    theta: the two-level theta-scheme of Eq. (GCN) with this theta (MMFD_FLAG_THETA); None: the
    explicit scheme.
    boundary: "periodic" or "dirichlet" (prescribed values on the outermost ring of nodes).
    """
    d = mmfd_desc_init()
    d.pde = PDE[pde]
    d.lattice = LATTICE[lattice]
    d.levels = int(levels)
    d.dim = 2 if lattice.startswith("D2") else 3
    nn = list(n) + [1] * (3 - len(n))
    for i in range(3):
        d.n[i] = int(nn[i])
    d.dt = float(dt)
    for i, v in enumerate(dx):
        d.dx[i] = float(v)
    if d0 is not None:
        for i, v in enumerate(d0):
            d.d0[i] = float(v)
    if K is not None:
        K = np.asarray(K, dtype=float)
        for i in range(K.shape[0]):
            for j in range(K.shape[1]):
                d.K[i][j] = float(K[i, j])
    if u is not None:
        for i, v in enumerate(u):
            d.u[i] = float(v)
    d.lambda_bar = float(lambda_bar)
    if flux is not None:
        for i, row in enumerate(flux):
            for j, v in enumerate(row):
                d.flux[i][j] = float(v)
    if diff is not None:
        for j, v in enumerate(diff):
            d.diff[j] = float(v)
    d.rho0 = float(rho0)
    if a is not None:
        d.coef_mode = MMFD_COEF_EXPLICIT
        for i in range(3):
            d.a[i] = float(a[i])
            d.ahat[i] = float(ahat[i]) if ahat is not None else 0.0
            d.abar[i] = float(abar[i]) if abar is not None else float(a[i])
            d.abarhat[i] = float(abarhat[i]) if abarhat is not None else (float(ahat[i]) if ahat is not None else 0.0)
    else:
        d.coef_mode = MMFD_COEF_TARGETS
        if targets is not None:
            for i, v in enumerate(targets):
                d.targets[i] = float(v)
        tb = targets_bar if targets_bar is not None else targets
        if tb is not None:
            for i, v in enumerate(tb):
                d.targets_bar[i] = float(v)
    d.storage = STORAGE[storage]
    d.flags = int(flags)
    if sets:
        d.flags |= MMFD_FLAG_TWO_SETS
        for name in ("d2", "d1", "bar_d2", "bar_d1"):
            lv = sets.get(name, ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)))
            arr = getattr(d, name)
            for l in range(2):
                for k in range(3):
                    arr[l][k] = float(lv[l][k])
    if ref is not None:
        for i, v in enumerate(ref):
            d.ref[i] = float(v)
    d.temporal_depth = int(temporal_depth)
    d.source = SOURCE[source]
    for i in range(3):
        d.b[i] = float(b[i]) if b is not None else 0.0
        d.bhat[i] = float(bhat[i]) if bhat is not None else 0.0
    if theta is not None:
        d.flags |= MMFD_FLAG_THETA
        d.theta = float(theta)
    d.boundary = {"periodic": MMFD_BC_PERIODIC, "dirichlet": MMFD_BC_DIRICHLET}[boundary]
    if seed is not None:
        d.seed = int(seed)
    if stream is not None:
        d.stream = stream
    return d


# ------------------------------------------------------------------ torch-backed solver object

class _TorchAllocator:
    """Device memory for the library's level buffers from torch's caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, out_ptr, ctx):
        try:
            p = self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return -1
        self.live[p] = nbytes
        out_ptr[0] = p
        return 0

    def _free(self, ptr, ctx):
        if ptr in self.live:
            del self.live[ptr]
            self.torch.cuda.caching_allocator_delete(ptr)


class Solver:
    """A created MMFD solver; fields move as numpy arrays (host) or torch tensors (device)."""

    def __init__(self, desc: mmfd_desc, use_torch_allocator: bool = True, stream=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device()
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream_obj = s
        self.stream = s.cuda_stream
        desc.stream = self.stream
        self._alloc = None
        if use_torch_allocator:
            self._alloc = _TorchAllocator(self.device, self.stream)
            desc.alloc = self._alloc.alloc_cb
            desc.free_fn = self._alloc.free_cb
        self.desc = desc
        self.h = mmfd_create(desc)
        self.info = mmfd_get_info(self.h)
        self.nf = self.info.nf
        self.dim = desc.dim
        self.shape = (desc.n[1], desc.n[0]) if desc.dim == 2 else (desc.n[2], desc.n[1], desc.n[0])

    def close(self):
        if self.h:
            mmfd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, fields, level: int = 0):
        """fields: nf numpy arrays (host, float64/float32) or CUDA torch tensors."""
        t = self.torch
        if len(fields) != self.nf:
            raise ValueError(f"expected {self.nf} fields")
        if isinstance(fields[0], t.Tensor) and fields[0].is_cuda:
            ts = [f.contiguous() for f in fields]
            dtype = MMFD_DT_F64 if ts[0].dtype == t.float64 else MMFD_DT_F32
            ts = [f.to(t.float64 if dtype == MMFD_DT_F64 else t.float32) for f in ts]
            mmfd_set_fields(self.h, level, [f.data_ptr() for f in ts], MMFD_DEVICE, dtype)
            self._keep = ts
        else:
            arrs = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
            mmfd_set_fields(self.h, level, [a.ctypes.data for a in arrs], MMFD_HOST, MMFD_DT_F64)

    def set_source(self, fields, level: int = 0):
        """Source fields (S, then the M_1F components for source "sm"): numpy arrays (host) or
        CUDA torch tensors."""
        t = self.torch
        if fields and isinstance(fields[0], t.Tensor) and fields[0].is_cuda:
            f32 = all(f.dtype == t.float32 and f.is_contiguous() for f in fields)
            ts = list(fields) if f32 else [f.contiguous().to(t.float64) for f in fields]
            mmfd_set_source(self.h, level, [f.data_ptr() for f in ts], MMFD_DEVICE,
                            MMFD_DT_F32 if f32 else MMFD_DT_F64)
            self._keep_src = ts
        else:
            arrs = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
            mmfd_set_source(self.h, level, [a.ctypes.data for a in arrs], MMFD_HOST, MMFD_DT_F64)

    def set_boundary(self, fields):
        """Dirichlet solvers: boundary values for the following steps, as full fields (numpy
        arrays on the host or CUDA torch tensors) of which the boundary nodes are used."""
        t = self.torch
        if fields and isinstance(fields[0], t.Tensor) and fields[0].is_cuda:
            f32 = all(f.dtype == t.float32 and f.is_contiguous() for f in fields)
            ts = list(fields) if f32 else [f.contiguous().to(t.float64) for f in fields]
            mmfd_set_boundary(self.h, [f.data_ptr() for f in ts], MMFD_DEVICE, MMFD_DT_F32 if f32 else MMFD_DT_F64)
            self._keep_bnd = ts
        else:
            arrs = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
            mmfd_set_boundary(self.h, [a.ctypes.data for a in arrs], MMFD_HOST, MMFD_DT_F64)

    def step(self, nsteps: int = 1):
        mmfd_step(self.h, nsteps)

    def fields(self, level: int = 0, device: bool = False, dtype=np.float64):
        if device:
            t = self.torch
            tdt = t.float64 if dtype == np.float64 else t.float32
            outs = [t.empty(self.shape, dtype=tdt, device="cuda") for _ in range(self.nf)]
            mmfd_fields(self.h, level, [o.data_ptr() for o in outs], MMFD_DEVICE,
                        MMFD_DT_F64 if dtype == np.float64 else MMFD_DT_F32)
            return outs
        outs = [np.empty(self.shape, dtype=dtype) for _ in range(self.nf)]
        mmfd_fields(self.h, level, [o.ctypes.data for o in outs], MMFD_HOST,
                    MMFD_DT_F64 if dtype == np.float64 else MMFD_DT_F32)
        return outs

    def reduce(self, what: int = MMFD_RED_SUM):
        return mmfd_reduce(self.h, what, 1 if what == MMFD_RED_NONFINITE else self.nf)

    def error_norms(self, ref: np.ndarray, field: int = 0):
        r = np.ascontiguousarray(ref, dtype=np.float64)
        return mmfd_error_norms(self.h, field, r.ctypes.data, MMFD_HOST, MMFD_DT_F64)

    def get_info(self) -> mmfd_info_t:
        return mmfd_get_info(self.h)

    def autotune(self, cache_path: Optional[str] = None) -> mmfd_tune_info:
        return mmfd_autotune(self.h, cache_path)


def info_dict(info: mmfd_info_t) -> dict:
    out = {}
    for name, _ in info._fields_:
        v = getattr(info, name)
        if hasattr(v, "__len__"):
            try:
                v = [list(x) if hasattr(x, "__len__") else x for x in v]
            except TypeError:
                pass
        out[name] = v
    return out


# ------------------------------------------------------------------ solve server

def mmfd_server_create(hbm_budget: int, max_slots: int = 64, steps_per_tick: int = 16, use_graphs: bool = True,
                       stream: Optional[int] = None) -> int:
    d = mmfd_server_desc()
    d.hbm_budget = int(hbm_budget)
    d.max_slots = int(max_slots)
    d.steps_per_tick = int(steps_per_tick)
    d.use_graphs = 1 if use_graphs else 0
    d.stream = stream
    h = C.c_void_p()
    check(lib.mmfd_server_create(C.byref(d), C.byref(h)), "mmfd_server_create")
    return h.value


def mmfd_submit(srv: int, d: mmfd_desc, ptrs: Sequence[int], dtype: int, nsteps: int) -> int:
    t = C.c_ulonglong()
    check(lib.mmfd_submit(srv, C.byref(d), _ptr_array(ptrs), dtype, int(nsteps), C.byref(t)), "mmfd_submit")
    return t.value


def mmfd_poll(srv: int, ticket: int):
    r = mmfd_result()
    rc = lib.mmfd_poll(srv, ticket, C.byref(r))
    if rc < 0:
        raise MMFDError(rc, "mmfd_poll")
    return rc, r


def mmfd_server_drain(srv: int) -> None:
    check(lib.mmfd_server_drain(srv), "mmfd_server_drain")


def mmfd_result_fields(srv: int, ticket: int, ptrs: Sequence[int], where: int, dtype: int) -> None:
    check(lib.mmfd_result_fields(srv, ticket, _ptr_array(ptrs), where, dtype), "mmfd_result_fields")


def mmfd_release(srv: int, ticket: int) -> None:
    check(lib.mmfd_release(srv, ticket), "mmfd_release")


def mmfd_server_get_stats(srv: int) -> mmfd_server_stats:
    s = mmfd_server_stats()
    check(lib.mmfd_server_get_stats(srv, C.byref(s)), "mmfd_server_get_stats")
    return s


def mmfd_server_destroy(srv: int) -> None:
    check(lib.mmfd_server_destroy(srv), "mmfd_server_destroy")


class Server:
    """A solve server; requests go in as numpy fields, results come out as numpy fields."""

    def __init__(self, hbm_budget: int, max_slots: int = 64, steps_per_tick: int = 16, use_graphs: bool = True,
                 stream=None):
        self.stream_obj = stream
        sp = stream.cuda_stream if stream is not None else None
        self.h = mmfd_server_create(hbm_budget, max_slots, steps_per_tick, use_graphs, sp)
        self.meta = {}

    def submit(self, desc: mmfd_desc, fields, nsteps: int) -> int:
        arrs = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
        t = mmfd_submit(self.h, desc, [a.ctypes.data for a in arrs], MMFD_DT_F64, nsteps)
        shape = arrs[0].shape
        self.meta[t] = (len(arrs), shape)
        return t

    def poll(self, ticket: int):
        return mmfd_poll(self.h, ticket)

    def drain(self):
        mmfd_server_drain(self.h)

    def result(self, ticket: int):
        nf, shape = self.meta[ticket]
        outs = [np.empty(shape, dtype=np.float64) for _ in range(nf)]
        mmfd_result_fields(self.h, ticket, [o.ctypes.data for o in outs], MMFD_HOST, MMFD_DT_F64)
        return outs

    def release(self, ticket: int):
        mmfd_release(self.h, ticket)
        self.meta.pop(ticket, None)

    def stats(self) -> dict:
        s = mmfd_server_get_stats(self.h)
        return {name: getattr(s, name) for name, _ in s._fields_}

    def close(self):
        if self.h:
            mmfd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
