"""Python access to the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the cpu_baseline /
``--impl reference`` legs of ``bench.py`` may import this module.  It never
imports the CUDA package and the CUDA package never imports it.

Fields are numpy float64 arrays; a level is a list of ``nf`` arrays of shape
(ny, nx) or (nz, ny, nx), x fastest.  LCDE/NCDE: nf = 1 (phi).  NSE:
nf = 1 + dim (rho, u_x, u_y[, u_z]).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SRC = os.path.join(HERE, "mmfd_oracle.c")

LATTICES = {"D2Q5": 0, "D2Q9": 1, "D3Q7": 2, "D3Q19": 3}
PDES = {"LCDE": 0, "NCDE": 1, "NSE": 2}
FORMS = {"mesofd": 1, "mmfd": 2, "central": 3, "mesofd_trt": 4}
SOURCES = {"none": 0, "s": 1, "su": 2, "sm": 3}
LATTICE_DIM = {"D2Q5": 2, "D2Q9": 2, "D3Q7": 3, "D3Q19": 3}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP over nodes only)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
           "-shared", "-fPIC", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("pde", C.c_int), ("levels", C.c_int),
        ("n", C.c_int * 3), ("c", C.c_double * 3), ("d0", C.c_double * 3),
        ("a", C.c_double * 3), ("ahat", C.c_double * 3),
        ("abar", C.c_double * 3), ("abarhat", C.c_double * 3),
        ("u", C.c_double * 3), ("Cmat", C.c_double * 9),
        ("flux", C.c_double * 12), ("m2", C.c_double * 5), ("rho0", C.c_double),
        ("two_sets", C.c_int),
        ("d2", (C.c_double * 3) * 2), ("d1", (C.c_double * 3) * 2),
        ("bar_d2", (C.c_double * 3) * 2), ("bar_d1", (C.c_double * 3) * 2),
        ("dt", C.c_double), ("src_mode", C.c_int), ("b", C.c_double * 3), ("bhat", C.c_double * 3),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            dp = C.POINTER(C.c_double)
            pp = C.POINTER(_Problem)
            L.or_lattice.argtypes = [C.c_int, dp, dp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), dp, dp]
            L.or_geq.argtypes = [C.c_int, dp, dp, C.c_double, dp, dp, dp]
            L.or_feq.argtypes = [pp, dp, dp]
            L.or_set_threads.argtypes = [C.c_int]
            L.or_step.argtypes = [pp, C.c_int, dp, dp, dp]
            L.or_step_nodes.argtypes = [pp, C.c_int, dp, dp, C.POINTER(C.c_longlong), C.c_longlong, dp]
            L.or_step_src.argtypes = [pp, C.c_int, dp, dp, dp, dp, dp]
            L.or_step_nodes_src.argtypes = [pp, C.c_int, dp, dp, dp, dp, C.POINTER(C.c_longlong), C.c_longlong, dp]
            L.or_run.argtypes = [pp, C.c_int, C.c_longlong, dp, dp]
            L.or_lbgk_tau1_run.argtypes = [pp, C.c_longlong, dp]
            L.or_trt_run.argtypes = [pp, C.c_double, C.c_longlong, dp]
            _lib = L
        return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr3(v, n=3):
    out = [0.0] * n
    for i, x in enumerate(v):
        out[i] = float(x)
    return out


@dataclass
class Problem:
    """A problem in the paper's notation (all scheme and EDF parameters explicit).

    a, ahat, abar, abarhat: coefficient triples (a_{-1}, a_0, a_1).
    sets: None for the one-set scheme, or the multiple-parameter-set scheme of Eq. (2-2-1b) as
    a dict of triples per level ((level t, level t - dt)): "d2" (second-difference term on
    f^eq,+ of the phi / rho moment), "d1" (first-difference term on f^eq,-), and for the NSE
    momentum "bar_d2" (second difference on f^eq,-) and "bar_d1" (first difference on f^eq,+).
    a / ahat (abar / abarhat) keep the zeroth-order term.
    source: "none", or the source distribution F_j = g_j^eq(S, M_1F, 0) of Eq. (SourceF) with
    M_1F = 0 ("s"), M_1F = S u ("su", LCDE: the F_j of Example 1) or M_1F given as fields
    ("sm"); b / bhat: the b_k of level t and t - dt (Eq. (2-1) / (3layer-1)); dt: the time step
    that multiplies them.
    """
    lattice: str
    pde: str
    levels: int
    n: Sequence[int]
    c: Sequence[float]
    d0: Sequence[float]
    a: Sequence[float]
    ahat: Sequence[float] = (0.0, 0.0, 0.0)
    abar: Sequence[float] = (0.0, 0.0, 0.0)
    abarhat: Sequence[float] = (0.0, 0.0, 0.0)
    u: Sequence[float] = (0.0, 0.0, 0.0)
    Cmat: Sequence[float] = field(default_factory=lambda: [0.0] * 9)
    flux: Sequence[float] = field(default_factory=lambda: [0.0] * 12)
    m2: Sequence[float] = field(default_factory=lambda: [0.0] * 5)
    rho0: float = 1.0
    sets: Optional[dict] = None
    dt: float = 0.0
    source: str = "none"
    b: Sequence[float] = (0.0, 0.0, 0.0)
    bhat: Sequence[float] = (0.0, 0.0, 0.0)

    @property
    def dim(self) -> int:
        return LATTICE_DIM[self.lattice]

    @property
    def nf(self) -> int:
        return 1 + self.dim if self.pde == "NSE" else 1

    @property
    def nsrc(self) -> int:
        return {"none": 0, "s": 1, "su": 1, "sm": 1 + self.dim}[self.source]

    @property
    def shape(self):
        nx, ny, nz = (list(self.n) + [1, 1])[:3]
        return (ny, nx) if self.dim == 2 else (nz, ny, nx)

    def to_c(self) -> _Problem:
        p = _Problem()
        p.lattice = LATTICES[self.lattice]
        p.pde = PDES[self.pde]
        p.levels = int(self.levels)
        n = (list(self.n) + [1, 1])[:3]
        p.n = (C.c_int * 3)(*[int(x) for x in n])
        p.c = (C.c_double * 3)(*_arr3(self.c))
        p.d0 = (C.c_double * 3)(*_arr3(self.d0))
        for name in ("a", "ahat", "abar", "abarhat", "u"):
            setattr(p, name, (C.c_double * 3)(*_arr3(getattr(self, name))))
        p.Cmat = (C.c_double * 9)(*_arr3(np.asarray(self.Cmat, dtype=float).ravel(), 9))
        p.flux = (C.c_double * 12)(*_arr3(np.asarray(self.flux, dtype=float).ravel(), 12))
        p.m2 = (C.c_double * 5)(*_arr3(self.m2, 5))
        p.rho0 = float(self.rho0)
        if self.sets:
            p.two_sets = 1
            for name in ("d2", "d1", "bar_d2", "bar_d1"):
                lv = self.sets.get(name, ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)))
                arr = getattr(p, name)
                for l in range(2):
                    arr[l] = (C.c_double * 3)(*_arr3(lv[l]))
        p.dt = float(self.dt)
        p.src_mode = SOURCES[self.source]
        p.b = (C.c_double * 3)(*_arr3(self.b))
        p.bhat = (C.c_double * 3)(*_arr3(self.bhat))
        return p


def _pack(level: Sequence[np.ndarray], nf: int, shape) -> np.ndarray:
    if len(level) != nf:
        raise ValueError(f"expected {nf} fields, got {len(level)}")
    out = np.empty((nf,) + tuple(shape), dtype=np.float64)
    for i, f in enumerate(level):
        f = np.asarray(f, dtype=np.float64)
        if f.shape != tuple(shape):
            raise ValueError(f"field {i} has shape {f.shape}, expected {shape}")
        out[i] = f
    return np.ascontiguousarray(out)


def _unpack(buf: np.ndarray) -> List[np.ndarray]:
    return [buf[i].copy() for i in range(buf.shape[0])]


def set_threads(n: int) -> int:
    return lib().or_set_threads(int(n))


def lattice(name: str, d0: Sequence[float], c: Sequence[float]):
    """(e, w, cs2) of App. A: e is (b, 3) int, w (b,), cs2 (3,)."""
    dim = C.c_int()
    b = C.c_int()
    e = (C.c_int * 57)()
    w = np.zeros(19)
    cs2 = np.zeros(3)
    d0a = np.array(_arr3(d0))
    ca = np.array(_arr3(c))
    rc = lib().or_lattice(LATTICES[name], _dp(d0a), _dp(ca), C.byref(dim), C.byref(b), e, _dp(w), _dp(cs2))
    if rc != 0:
        raise ValueError("bad lattice")
    E = np.array(e[: 3 * b.value], dtype=np.int64).reshape(b.value, 3)
    return E, w[: b.value].copy(), cs2


def geq(name: str, d0, c, A: float, B, Cm) -> np.ndarray:
    """g^eq(A, B, C) of Eq. (3-3) for every direction."""
    g = np.zeros(19)
    d0a = np.array(_arr3(d0))
    ca = np.array(_arr3(c))
    Ba = np.array(_arr3(B))
    Ca = np.array(_arr3(np.asarray(Cm, dtype=float).ravel(), 9))
    rc = lib().or_geq(LATTICES[name], _dp(d0a), _dp(ca), float(A), _dp(Ba), _dp(Ca), _dp(g))
    if rc != 0:
        raise ValueError("bad lattice")
    E, _, _ = lattice(name, d0, c)
    return g[: E.shape[0]].copy()


def feq(prob: Problem, node_fields: Sequence[float]) -> np.ndarray:
    f = np.array(_arr3(node_fields, 4))
    out = np.zeros(19)
    p = prob.to_c()
    if lib().or_feq(C.byref(p), _dp(f), _dp(out)) != 0:
        raise ValueError("bad problem")
    E, _, _ = lattice(prob.lattice, prob.d0, prob.c)
    return out[: E.shape[0]].copy()


def _pack_src(prob: Problem, src):
    """(level t, level t - dt) source fields -> two packed buffers (or None)."""
    if prob.source == "none":
        return None, None
    if src is None:
        raise ValueError("this problem has source terms: pass src=(fields at t, fields at t - dt)")
    s0 = _pack(src[0], prob.nsrc, prob.shape)
    s1 = _pack(src[1], prob.nsrc, prob.shape) if (len(src) > 1 and src[1] is not None) else np.zeros_like(s0)
    return s0, s1


def _ptr(b):
    return _dp(b) if b is not None else None


def step(prob: Problem, level_n: Sequence[np.ndarray], level_nm1: Optional[Sequence[np.ndarray]] = None,
         form: str = "mmfd", src=None) -> List[np.ndarray]:
    """One explicit MMFD step; returns the new level as a list of fields.

    src: for problems with source terms, (source fields at t, source fields at t - dt), each a
    list of prob.nsrc arrays (the second may be None for two-level problems)."""
    bn = _pack(level_n, prob.nf, prob.shape)
    bm = _pack(level_nm1, prob.nf, prob.shape) if level_nm1 is not None else np.zeros_like(bn)
    s0, s1 = _pack_src(prob, src)
    out = np.empty_like(bn)
    p = prob.to_c()
    rc = lib().or_step_src(C.byref(p), FORMS[form], _dp(bn), _dp(bm), _ptr(s0), _ptr(s1), _dp(out))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return _unpack(out)


def step_nodes(prob: Problem, level_n, level_nm1, nodes: np.ndarray, form: str = "mmfd", src=None) -> np.ndarray:
    """Outputs of one step at the given flat node indices; returns (count, nf)."""
    bn = _pack(level_n, prob.nf, prob.shape)
    bm = _pack(level_nm1, prob.nf, prob.shape) if level_nm1 is not None else np.zeros_like(bn)
    s0, s1 = _pack_src(prob, src)
    idx = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.empty((idx.size, prob.nf))
    p = prob.to_c()
    rc = lib().or_step_nodes_src(C.byref(p), FORMS[form], _dp(bn), _dp(bm), _ptr(s0), _ptr(s1),
                                 idx.ctypes.data_as(C.POINTER(C.c_longlong)), idx.size, _dp(out))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return out


def run_source(prob: Problem, level_n, level_nm1, nsteps: int, source, form: str = "mmfd"):
    """nsteps steps of a problem with source terms; source(m) gives the source fields at time
    t0 + m dt (m = 0 is the time of level_n, m = -1 that of level_nm1).  Returns (level at the
    end, level before it)."""
    cur = [np.asarray(f, dtype=np.float64) for f in level_n]
    prev = [np.asarray(f, dtype=np.float64) for f in level_nm1] if level_nm1 is not None else None
    for m in range(int(nsteps)):
        new = step(prob, cur, prev, form=form, src=(source(m), source(m - 1)))
        prev, cur = cur, new
    return cur, (prev if prob.levels == 3 else None)


def run(prob: Problem, level_n, level_nm1=None, nsteps: int = 1, form: str = "mmfd"):
    """nsteps steps; returns (level at the end, level before it)."""
    bn = _pack(level_n, prob.nf, prob.shape)
    if prob.levels == 3:
        if level_nm1 is None:
            raise ValueError("three-level runs need the level t - dt")
        bm = _pack(level_nm1, prob.nf, prob.shape)
    else:
        bm = np.zeros_like(bn)
    p = prob.to_c()
    rc = lib().or_run(C.byref(p), FORMS[form], int(nsteps), _dp(bn), _dp(bm))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return _unpack(bn), (_unpack(bm) if prob.levels == 3 else None)


def theta_operator_symbol(prob: Problem, form: str = "mmfd") -> np.ndarray:
    """Eigenvalues ell of the difference operator L of the two-level LCDE scheme on the grid.

    The explicit update Eq. (2-2-2) without sources is phi + L phi: the zeroth-order term is
    sum_k a_k phi = phi (A_00 = 1) and L collects the central differences of Eq. (2-2-1).  For the
    LCDE L is linear and shift-invariant on the periodic grid, i.e. circulant: L phi = h * phi
    (circular convolution) with the impulse response h = L delta_0, so L is diagonalised by the
    DFT with eigenvalues DFT(h) (numpy axis order)."""
    if prob.pde != "LCDE" or prob.levels != 2:
        raise ValueError("the theta-scheme is defined here for the two-level LCDE")
    delta = np.zeros(prob.shape)
    delta[(0,) * len(prob.shape)] = 1.0
    h = step(prob, [delta], form=form)[0] - delta
    return np.fft.fftn(h)


def theta_run(prob: Problem, level_n, nsteps: int, theta: float, form: str = "mmfd") -> List[np.ndarray]:
    """nsteps steps of the two-level theta-scheme Eq. (GCN) for the LCDE without sources.

    Eq. (GCN) weights the difference terms of level t - dt by theta and those of the new level t
    by theta_1 = 1 - theta: phi^{n+1} = phi^n + theta L phi^n + theta_1 L phi^{n+1}, i.e. the
    linear system (I - theta_1 L) phi^{n+1} = (I + theta L) phi^n.  theta = 1 is the explicit
    scheme Eq. (2-2-2), theta = 0 the implicit one Eq. (2-2-3).  Each step solves the system
    exactly in the DFT basis of the circulant L (theta_operator_symbol)."""
    if not 0.0 <= theta <= 1.0:
        raise ValueError("theta must lie in [0, 1]")
    ell = theta_operator_symbol(prob, form)
    den = 1.0 - (1.0 - theta) * ell
    if np.abs(den).min() == 0.0:
        raise ValueError("I - (1 - theta) L is singular on this grid")
    mult = (1.0 + theta * ell) / den
    phi = np.asarray(level_n[0], dtype=np.float64)
    for _ in range(int(nsteps)):
        phi = np.real(np.fft.ifftn(np.fft.fftn(phi) * mult))
    return [phi]


def lbgk_tau1_run(prob: Problem, level_n, nsteps: int) -> List[np.ndarray]:
    """Collide-and-stream LBGK with tau = 1 on explicit populations (independent check)."""
    b = _pack(level_n, prob.nf, prob.shape)
    p = prob.to_c()
    if lib().or_lbgk_tau1_run(C.byref(p), int(nsteps), _dp(b)) != 0:
        raise ValueError("oracle rejected the problem")
    return _unpack(b)


def trt_run(prob: Problem, level_n, s_minus: float, nsteps: int) -> List[np.ndarray]:
    """Independent TRT lattice-Boltzmann run (s+ = 2 - s-), from equilibrium populations of
    level_n; returns the moments after nsteps."""
    buf = _pack(level_n, prob.nf, prob.shape)
    p = prob.to_c()
    rc = lib().or_trt_run(C.byref(p), float(s_minus), int(nsteps), _dp(buf))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return _unpack(buf)


class LevelStepper:
    """Pack one level once, then advance it in place by whole oracle steps (used to time full
    steps of a large workload without unpacking between them)."""

    def __init__(self, prob: Problem, level_n, level_nm1=None, form: str = "mmfd"):
        self.prob = prob
        self.p = prob.to_c()
        self.bn = _pack(level_n, prob.nf, prob.shape)
        self.bm = _pack(level_nm1, prob.nf, prob.shape) if level_nm1 is not None else np.zeros_like(self.bn)
        self.form = FORMS[form]

    def step(self, nsteps: int = 1) -> None:
        rc = lib().or_run(C.byref(self.p), self.form, int(nsteps), _dp(self.bn), _dp(self.bm))
        if rc != 0:
            raise ValueError("oracle rejected the problem")

    def level(self):
        return _unpack(self.bn)


class NodeSampler:
    """Pack one level once, then evaluate the oracle step on contiguous node ranges.

    Used to time the oracle on a bounded sample of a large workload (the per-node work is
    exactly that of a full step; only the set of nodes is bounded)."""

    def __init__(self, prob: Problem, level_n, level_nm1=None, form: str = "mmfd"):
        self.prob = prob
        self.p = prob.to_c()
        self.bn = _pack(level_n, prob.nf, prob.shape)
        self.bm = _pack(level_nm1, prob.nf, prob.shape) if level_nm1 is not None else np.zeros_like(self.bn)
        self.form = FORMS[form]
        self.N = int(np.prod(prob.shape))

    def run(self, start: int, count: int) -> np.ndarray:
        idx = (np.arange(count, dtype=np.int64) + int(start)) % self.N
        out = np.empty((count, self.prob.nf))
        rc = lib().or_step_nodes(C.byref(self.p), self.form, _dp(self.bn), _dp(self.bm),
                                 idx.ctypes.data_as(C.POINTER(C.c_longlong)), count, _dp(out))
        if rc != 0:
            raise ValueError("oracle rejected the problem")
        return out
