"""ctypes binding of ``libofks.so`` (names mirror ``include/ofks.h``).

Argument marshalling only: every computation runs in the library's CUDA kernels.  Loading
fails loudly when the shared library is missing or cannot be opened; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libofks.so")

OK, EINVAL, ECUDA, ENOMEM, ESTATE, ENOTCONV, ENONFINITE, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
PC = {"none": 0, "pcg": 1, "exact": 2, "learned": 3}
PRECISION = {"fp64": 0, "mixed": 1}
ETA = {"bb2": 0, "bb1": 1, "abb1": 2, "abb2": 3, "bb2_raw": 4, "fixed": 5}
METHOD = {"pcal": 0, "plam": 1, "moptqr": 2}
HPC = {"jacobi": 0, "multigrid": 1, "separable": 2}        # Hartree CG preconditioners
HPC_NAMES = {v: k for k, v in HPC.items()}
FIELDS = {"rho_q": 0, "vh_q": 1, "vxc_q": 2, "exc_q": 3, "U": 4, "HX": 5, "BX": 6, "G": 7, "D": 8,
          "Lambda0": 9, "S": 10, "Lambda": 11, "vext_q": 12}
MATS = {"L": 0, "B": 1, "H": 2}
PCGPC = {"jacobi": 0, "separable": 1}
STATIC_NUCLEI_MAX = 1024          # OFKS_STATIC_NUCLEI_MAX
SYMBOLS = ("ofks_default_params", "ofks_create", "ofks_destroy", "ofks_last_error", "ofks_set_mesh",
           "ofks_set_nuclei", "ofks_set_nuclei_static", "ofks_set_params", "ofks_init_orbitals", "ofks_set_orbitals",
           "ofks_get_orbitals", "ofks_step", "ofks_solve", "ofks_evaluate", "ofks_rayleigh_ritz",
           "ofks_get_field", "ofks_apply", "ofks_get_sizes", "ofks_poisson_info", "ofks_fma_peak", "ofks_get_history", "ofks_save_state",
           "ofks_load_state", "ofks_profile", "ofks_profile_get", "ofks_precond_init", "ofks_precond_get_weights",
           "ofks_precond_set_weights", "ofks_precondition", "ofks_train_precond_step", "ofks_precond_grads",
           "ofks_record_pair", "ofks_train_precond", "ofks_train_info")


class OfksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ofks error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("p", C.c_int32), ("beta", C.c_double), ("occ", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("precision", C.c_int32), ("precond", C.c_int32),
                ("pcg_iters", C.c_int32), ("eta_rule", C.c_int32), ("eta_fixed", C.c_double),
                ("eta_min", C.c_double), ("eta_max", C.c_double), ("hartree", C.c_int32),
                ("xc", C.c_int32), ("multipole_lmax", C.c_int32), ("poisson_tol", C.c_double),
                ("poisson_max_iter", C.c_int32), ("poisson_pc", C.c_int32), ("mixed_tol", C.c_double),
                ("poisson_tol_mixed", C.c_double), ("judge_tau", C.c_double), ("learned_tc", C.c_int32),
                ("poisson_adaptive", C.c_int32), ("poisson_csr", C.c_int32),
                ("gram_tc", C.c_int32), ("spmm_f32_rows", C.c_int32), ("poisson_sep_tc", C.c_int32),
                ("pcg_compact", C.c_int32), ("cuda_graphs", C.c_int32), ("pcg_staged", C.c_int32),
                ("sweep_pc32", C.c_int32), ("method", C.c_int32), ("learned_loss", C.c_int32),
                ("learned_retry", C.c_int32), ("pcg_pc", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("e_total", C.c_double), ("e_nuc", C.c_double), ("kkt", C.c_double), ("fea", C.c_double),
                ("kkt0", C.c_double), ("eta", C.c_double), ("iters", C.c_int32), ("converged", C.c_int32),
                ("seconds", C.c_double), ("hartree_iters", C.c_int32), ("hartree_total", C.c_int32),
                ("switch_iter", C.c_int32), ("judge_accept", C.c_int64), ("judge_total", C.c_int64),
                ("active_last", C.c_int32), ("active_total", C.c_int64),
                ("pcg_cols_total", C.c_int64), ("learned_calls", C.c_int64), ("learned_warm", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def load(path: str = LIB_PATH):
    """Open libofks.so (once) and declare the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OfksError(ESTATE, f"{path} is missing: build it with paper_2007_14228_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "ofks_default_params": (None, [C.POINTER(Params)]),
        "ofks_create": (C.c_int, [C.POINTER(vp), C.c_int]),
        "ofks_destroy": (None, [vp]),
        "ofks_last_error": (C.c_char_p, [vp]),
        "ofks_set_mesh": (C.c_int, [vp, i64, _dp, i64, _ip, _up]),
        "ofks_set_nuclei": (C.c_int, [vp, i32, _dp, _dp]),
        "ofks_set_nuclei_static": (C.c_int, [vp, i32, _dp, _dp]),
        "ofks_set_params": (C.c_int, [vp, C.POINTER(Params)]),
        "ofks_init_orbitals": (C.c_int, [vp, _dp]),
        "ofks_set_orbitals": (C.c_int, [vp, _dp, i32]),
        "ofks_get_orbitals": (C.c_int, [vp, _dp]),
        "ofks_step": (C.c_int, [vp, i32, C.POINTER(Result)]),
        "ofks_solve": (C.c_int, [vp, C.POINTER(Result)]),
        "ofks_evaluate": (C.c_int, [vp, C.POINTER(Result)]),
        "ofks_rayleigh_ritz": (C.c_int, [vp, _dp]),
        "ofks_get_field": (C.c_int, [vp, i32, _dp, i64]),
        "ofks_apply": (C.c_int, [vp, i32, _dp, _dp, i32]),
        "ofks_get_sizes": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64),
                                     C.POINTER(i64)]),
        "ofks_poisson_info": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32),
                                        C.POINTER(i32)]),
        "ofks_fma_peak": (C.c_int, [vp, i32, C.POINTER(dbl)]),
        "ofks_get_history": (C.c_int, [vp, _dp, i32, C.POINTER(i32)]),
        "ofks_save_state": (C.c_int, [vp, C.c_char_p]),
        "ofks_load_state": (C.c_int, [vp, C.c_char_p]),
        "ofks_profile": (C.c_int, [vp, i32]),
        "ofks_profile_get": (C.c_int, [vp, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(C.c_char_p)]),
        "ofks_precond_init": (C.c_int, [vp, i32, C.c_uint64]),
        "ofks_precond_get_weights": (C.c_int, [vp, C.c_void_p, i64, C.POINTER(i64)]),
        "ofks_precond_set_weights": (C.c_int, [vp, _fp, i64]),
        "ofks_precondition": (C.c_int, [vp, i32, _dp, _dp, _dp]),
        "ofks_train_precond_step": (C.c_int, [vp, _dp, _dp, _dp, dbl, C.POINTER(dbl)]),
        "ofks_precond_grads": (C.c_int, [vp, _dp, _dp, _dp, _dp, i64, C.POINTER(dbl)]),
        "ofks_record_pair": (C.c_int, [vp, C.c_char_p, C.POINTER(i32)]),
        "ofks_train_precond": (C.c_int, [vp, C.c_char_p, i32, C.c_uint64]),
        "ofks_train_info": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_params(**overrides) -> Params:
    prm = Params()
    load().ofks_default_params(C.byref(prm))
    return updated_params(prm, **overrides)


def updated_params(base: Params, **overrides) -> Params:
    """A copy of `base` with the named fields replaced (enum fields also by name)."""
    prm = Params.from_buffer_copy(base)
    for k, v in overrides.items():
        if k == "precond" and isinstance(v, str):
            v = PC[v]
        if k == "eta_rule" and isinstance(v, str):
            v = ETA[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "poisson_pc" and isinstance(v, str):
            v = HPC[v]
        if k == "method" and isinstance(v, str):
            v = METHOD[v]
        if k == "pcg_pc" and isinstance(v, str):
            v = PCGPC[v]
        if isinstance(v, bool):
            v = int(v)
        setattr(prm, k, v)
    return prm


class Context:
    """One solver context on one CUDA device (``ofks_create`` .. ``ofks_destroy``)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.h = C.c_void_p()
        rc = self.lib.ofks_create(C.byref(self.h), int(device))
        if rc != OK:
            raise OfksError(rc, "ofks_create failed (no usable CUDA device?)")
        self.p = None
        self.n = None
        self._prm = None

    def close(self):
        if self.h:
            self.lib.ofks_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, rc):
        if rc != OK:
            raise OfksError(rc, self.lib.ofks_last_error(self.h).decode())
        return rc

    # ---- inputs
    def set_mesh(self, xyz, tet10, dirichlet):
        xyz = np.ascontiguousarray(xyz, np.float64)
        tet10 = np.ascontiguousarray(tet10, np.int64)
        dirichlet = np.ascontiguousarray(dirichlet, np.uint8)
        self._chk(self.lib.ofks_set_mesh(self.h, xyz.shape[0], xyz, tet10.shape[0], tet10, dirichlet))
        self.n = self.sizes()["n_free"]

    def set_nuclei(self, Z, R):
        Z = np.ascontiguousarray(Z, np.float64)
        R = np.ascontiguousarray(R, np.float64).reshape(-1, 3)
        self._chk(self.lib.ofks_set_nuclei(self.h, len(Z), Z, R))

    def set_nuclei_static(self, Z, R):
        """ofks_set_nuclei_static: same as set_nuclei, without any device allocation."""
        Z = np.ascontiguousarray(Z, np.float64)
        R = np.ascontiguousarray(R, np.float64).reshape(-1, 3)
        self._chk(self.lib.ofks_set_nuclei_static(self.h, len(Z), Z, R))

    def set_params(self, prm: Params | None = None, **overrides):
        """Set the parameters: `prm` with `overrides` applied, or, without `prm`, the parameters
        last set on this context (the defaults on the first call) with `overrides` applied."""
        if prm is None:
            prm = self._prm if self._prm is not None else default_params()
        prm = updated_params(prm, **overrides)
        self._chk(self.lib.ofks_set_params(self.h, C.byref(prm)))
        self._prm = prm
        self.p = prm.p

    def init_orbitals(self, V):
        V = np.ascontiguousarray(V, np.float64)
        self._check_block(V)
        self._chk(self.lib.ofks_init_orbitals(self.h, V))

    def set_orbitals(self, X, keep_history: bool = False):
        X = np.ascontiguousarray(X, np.float64)
        self._check_block(X)
        self._chk(self.lib.ofks_set_orbitals(self.h, X, int(keep_history)))

    def get_orbitals(self, out=None):
        out = np.empty((self.n, self.p)) if out is None else out
        self._chk(self.lib.ofks_get_orbitals(self.h, out))
        return out

    def _check_block(self, X):
        if X.shape != (self.n, self.p):
            raise OfksError(EINVAL, f"block shape {X.shape} != ({self.n}, {self.p})")

    # ---- iteration
    def step(self, k: int = 1) -> dict:
        r = Result()
        self._chk(self.lib.ofks_step(self.h, int(k), C.byref(r)))
        return r.as_dict()

    def solve(self, allow_notconv: bool = False) -> dict:
        r = Result()
        rc = self.lib.ofks_solve(self.h, C.byref(r))
        if rc != OK and not (allow_notconv and rc == ENOTCONV):
            self._chk(rc)
        return r.as_dict()

    def evaluate(self) -> dict:
        r = Result()
        self._chk(self.lib.ofks_evaluate(self.h, C.byref(r)))
        return r.as_dict()

    def rayleigh_ritz(self):
        eigs = np.empty(self.p)
        self._chk(self.lib.ofks_rayleigh_ritz(self.h, eigs))
        return eigs

    # ---- inspection
    def sizes(self) -> dict:
        v = [C.c_int64() for _ in range(5)]
        self._chk(self.lib.ofks_get_sizes(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("n_free", "n_nodes", "n_tets", "nnz", "nnz_full"), (x.value for x in v)))

    def fma_peak(self, bits: int = 64) -> float:
        """Measured FMA rate of the device in TFLOP/s (float64 or float32)."""
        t = C.c_double()
        self._chk(self.lib.ofks_fma_peak(self.h, PRECISION["fp64"] if bits == 64 else 32, C.byref(t)))
        return t.value

    def poisson_info(self) -> dict:
        fmt, stored, rows, pc = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
        lat = (C.c_int32 * 3)()
        self._chk(self.lib.ofks_poisson_info(self.h, C.byref(fmt), C.byref(stored), C.byref(rows), lat,
                                             C.byref(pc)))
        return {"format": "lattice" if fmt.value == 1 else "csr", "stored": stored.value, "rows": rows.value,
                "lattice": tuple(lat), "precond": HPC_NAMES[pc.value]}

    def get_field(self, name: str):
        s = self.sizes()
        which = FIELDS[name]
        if name.endswith("_q"):
            shape = (s["n_tets"], 4)
        elif name == "U":
            shape = (s["n_nodes"],)
        elif name in ("HX", "BX", "G", "D"):
            shape = (self.n, self.p)
        else:
            shape = (self.p, self.p)
        out = np.empty(shape)
        self._chk(self.lib.ofks_get_field(self.h, which, out, out.size))
        return out

    def apply(self, which: str, X):
        X = np.ascontiguousarray(X, np.float64)
        self._check_block(X)
        Y = np.empty_like(X)
        self._chk(self.lib.ofks_apply(self.h, MATS[which], X, Y, X.shape[1]))
        return Y

    def history(self, cap: int = 100000):
        buf = np.empty((cap, 6))
        n = C.c_int32()
        self._chk(self.lib.ofks_get_history(self.h, buf, cap, C.byref(n)))
        return buf[: n.value].copy()

    def save_state(self, path: str):
        self._chk(self.lib.ofks_save_state(self.h, path.encode()))

    def load_state(self, path: str):
        self._chk(self.lib.ofks_load_state(self.h, path.encode()))

    # ---- learned preconditioner
    def precond_init(self, width: int = 64, seed: int = 0):
        self._chk(self.lib.ofks_precond_init(self.h, int(width), int(seed)))

    def precond_get_weights(self):
        n = C.c_int64()
        self._chk(self.lib.ofks_precond_get_weights(self.h, None, 0, C.byref(n)))
        w = np.empty(n.value, np.float32)
        self._chk(self.lib.ofks_precond_get_weights(self.h, w.ctypes.data, n.value, C.byref(n)))
        return w

    def precond_set_weights(self, w):
        w = np.ascontiguousarray(w, np.float32)
        self._chk(self.lib.ofks_precond_set_weights(self.h, w, w.size))

    def precondition(self, mode: str, G, shifts):
        G = np.ascontiguousarray(G, np.float64)
        self._check_block(G)
        D = np.empty_like(G)
        self._chk(self.lib.ofks_precondition(self.h, PC[mode], G, np.ascontiguousarray(shifts, np.float64), D))
        return D

    def train_precond_step(self, G, shifts, Dstar, lr: float = 1e-3) -> float:
        loss = C.c_double()
        self._chk(self.lib.ofks_train_precond_step(self.h, np.ascontiguousarray(G, np.float64),
                                                   np.ascontiguousarray(shifts, np.float64),
                                                   np.ascontiguousarray(Dstar, np.float64), float(lr),
                                                   C.byref(loss)))
        return loss.value

    def precond_grads(self, G, shifts, Dstar):
        n = C.c_int64()
        self._chk(self.lib.ofks_precond_get_weights(self.h, None, 0, C.byref(n)))
        g = np.empty(n.value)
        loss = C.c_double()
        self._chk(self.lib.ofks_precond_grads(self.h, np.ascontiguousarray(G, np.float64),
                                              np.ascontiguousarray(shifts, np.float64),
                                              np.ascontiguousarray(Dstar, np.float64), g, g.size, C.byref(loss)))
        return loss.value, g

    def record_pair(self, path: str) -> int:
        """ofks_record_pair: append (G, shifts, T^{-1} G) at the current iterate to a pairs file;
        returns the number of columns with a negative shift."""
        act = C.c_int32()
        self._chk(self.lib.ofks_record_pair(self.h, path.encode(), C.byref(act)))
        return act.value

    def train_precond(self, path: str, epochs: int = 1, seed: int = 0):
        """ofks_train_precond: Adam over the pairs file in seeded shuffled order; returns
        (mean loss of the last epoch, Adam steps taken so far)."""
        self._chk(self.lib.ofks_train_precond(self.h, path.encode(), int(epochs), int(seed)))
        loss, steps = C.c_double(), C.c_int64()
        self._chk(self.lib.ofks_train_info(self.h, C.byref(loss), C.byref(steps)))
        return loss.value, steps.value

    def profile(self, on: bool):
        self._chk(self.lib.ofks_profile(self.h, int(on)))

    def profile_get(self) -> dict:
        out = {}
        for i in range(64):
            n, ms, name = C.c_int64(), C.c_double(), C.c_char_p()
            if self.lib.ofks_profile_get(self.h, i, C.byref(n), C.byref(ms), C.byref(name)) != OK:
                break
            out[name.value.decode()] = {"launches": n.value, "ms": ms.value}
        return out


def trained_weights():
    """The learned preconditioner's committed weights (see precond_weights.json for how they
    were trained)."""
    return np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "precond_weights.npy"))


def context_for(system, mesh, device: int = 0, **params) -> Context:
    """Context with mesh, nuclei and params of a synthetic ``inputs.System`` already set."""
    ctx = Context(device)
    ctx.set_mesh(mesh.xyz, mesh.tet10, mesh.dirichlet)
    ctx.set_nuclei(system.Z, system.R)
    kw = {"p": system.p, "occ": system.occ}
    kw.update(params)
    ctx.set_params(**kw)
    return ctx
