"""ctypes binding of libsu2dmrg (include/su2dmrg.h): argument marshalling only.

Every computation runs in the library (host tables in C++, the hot path in
CUDA kernels).  If the shared library is missing, loading raises; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsu2dmrg.so")

SU2_OK, SU2_EINVAL, SU2_ENOMEM, SU2_ECUDA, SU2_ETIMEOUT, SU2_ENOTCONV = range(6)
SU2_FP64, SU2_SPLIT_BF16, SU2_SPLIT_FP8 = 0, 1, 2   # FP8: reserved, rejected by the library
SU2_SITE_SPIN_HALF, SU2_SITE_ORBITAL = 0, 1
(SU2_MODEL_HEISENBERG, SU2_MODEL_QC_SKELETON, SU2_MODEL_CASIMIR_S2, SU2_MODEL_CASIMIR_N,
 SU2_MODEL_AB_INITIO) = range(5)

SYMBOLS = [
    "su2_ctx_create", "su2_ctx_destroy", "su2_last_error", "su2_ctx_status", "su2_ctx_wait", "su2_build_sectors", "su2_sectors_query",
    "su2_sectors_destroy", "su2_build_environment", "su2_env_query", "su2_env_tasks", "su2_env_terms", "su2_env_operator_block", "su2_env_destroy",
    "su2_apply_heff", "su2_apply_heff_host", "su2_apply_heff_static_scratch", "su2_diag_heff", "su2_davidson_create", "su2_davidson_step",
    "su2_davidson_solve", "su2_energy", "su2_energy_check", "su2_davidson_vector", "su2_davidson_destroy",
    "su2_profile_enable", "su2_profile_reset", "su2_profile_read", "su2_hash_group",
    "su2_sweep_create", "su2_sweep_run", "su2_sweep_checkpoint", "su2_sweep_destroy",
]


class Sector(C.Structure):
    _fields_ = [("N", C.c_int32), ("twoS", C.c_int32), ("dim", C.c_int32)]


class Block(C.Structure):
    _fields_ = [("a", C.c_int32), ("s1", C.c_int32), ("s2", C.c_int32), ("b", C.c_int32),
                ("jL1", C.c_int32), ("j2R", C.c_int32), ("rows", C.c_int32), ("cols", C.c_int32),
                ("offset", C.c_int64)]


class BondChain(C.Structure):
    _fields_ = [("n_bonds", C.c_int32), ("bond_offset", C.POINTER(C.c_int32)),
                ("sectors", C.POINTER(Sector))]


class Hamiltonian(C.Structure):
    _fields_ = [("model", C.c_int32), ("n_left", C.c_int32), ("n_right", C.c_int32),
                ("J", C.c_double), ("seed", C.c_uint64), ("h", C.c_void_p), ("eri", C.c_void_p),
                ("mps_left", C.c_void_p), ("mps_right", C.c_void_p)]


def _mps(a):
    """A float64 contiguous host copy of concatenated MPS tensors (or None)."""
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).ravel()


class EnvOpts(C.Structure):
    _fields_ = [("t_budget_bytes", C.c_int64), ("n_slices", C.c_int32), ("prepare_split", C.c_int32),
                ("autotune", C.c_int32), ("split_tol", C.c_double), ("shard_rank", C.c_int32),
                ("shard_count", C.c_int32), ("spin_limit", C.c_int32), ("resident_bytes", C.c_int64)]


class EnvInfo(C.Structure):
    _fields_ = [("psi_len", C.c_int64), ("n_blocks", C.c_int64), ("n_terms", C.c_int64),
                ("n_tasks", C.c_int64), ("n_k1", C.c_int64), ("n_chunks", C.c_int64),
                ("flops_su2", C.c_double), ("flops_u1_equiv", C.c_double), ("r_d", C.c_double),
                ("env_bytes", C.c_double), ("split_slices", C.c_int32), ("split_stage_k", C.c_int32),
                ("split_err_est", C.c_double), ("t_chunk_bytes", C.c_int64), ("renorm_flops", C.c_double),
                ("flops_u1_counted", C.c_double), ("r_cc", C.c_double), ("resident_bytes", C.c_int64),
                ("streamed_bytes", C.c_int64), ("n_io_chunks", C.c_int64)]


class SweepOpts(C.Structure):
    _fields_ = [("D", C.c_int32), ("prec", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("n_slices", C.c_int32), ("guess_seed", C.c_uint64), ("predict", C.c_int32), ("twoS", C.c_int32)]


class DavOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_sub", C.c_int32), ("keep", C.c_int32),
                ("max_iter", C.c_int32), ("prec", C.c_int32), ("use_graph", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsu2dmrg.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.su2_ctx_create.argtypes = [C.c_int, vp, C.POINTER(vp)]
        L.su2_ctx_destroy.argtypes = [vp]
        L.su2_last_error.argtypes = [vp]
        L.su2_last_error.restype = C.c_char_p
        L.su2_ctx_status.argtypes = [vp, C.POINTER(C.c_int32)]
        L.su2_ctx_wait.argtypes = [vp, C.c_double]
        L.su2_build_sectors.argtypes = [vp, C.POINTER(Sector), C.c_int32, C.POINTER(Sector), C.c_int32,
                                        C.c_int32, C.c_int32, C.c_int32, C.POINTER(vp)]
        L.su2_sectors_query.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                        C.POINTER(C.POINTER(Block))]
        L.su2_sectors_destroy.argtypes = [vp]
        L.su2_build_environment.argtypes = [vp, C.POINTER(Hamiltonian), C.POINTER(BondChain),
                                            C.POINTER(BondChain), vp, C.POINTER(EnvOpts), C.POINTER(vp)]
        L.su2_env_query.argtypes = [vp, C.POINTER(EnvInfo)]
        L.su2_env_tasks.argtypes = [vp, vp, vp, C.c_int64]
        L.su2_env_terms.argtypes = [vp, vp, vp, vp, vp, C.c_int64]
        L.su2_env_operator_block.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp,
                                             C.c_int32, C.c_int32]
        L.su2_env_destroy.argtypes = [vp]
        L.su2_apply_heff.argtypes = [vp, vp, vp, vp, C.c_int32]
        L.su2_apply_heff_host.argtypes = [vp, vp, vp, vp, C.c_int32]
        L.su2_apply_heff_static_scratch.argtypes = [vp, vp, vp, vp]
        L.su2_diag_heff.argtypes = [vp, vp, vp]
        L.su2_davidson_create.argtypes = [vp, vp, vp, C.POINTER(DavOpts), C.POINTER(vp)]
        L.su2_davidson_step.argtypes = [vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.su2_davidson_solve.argtypes = [vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int32)]
        L.su2_energy.argtypes = [vp, C.POINTER(C.c_double)]
        L.su2_davidson_vector.argtypes = [vp, vp, vp]
        L.su2_energy_check.argtypes = [vp, vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.su2_davidson_destroy.argtypes = [vp]
        L.su2_profile_enable.argtypes = [vp, C.c_int32]
        L.su2_profile_reset.argtypes = [vp]
        L.su2_profile_read.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_char_p)]
        L.su2_hash_group.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.POINTER(C.c_int64)]
        L.su2_sweep_create.argtypes = [vp, C.POINTER(Hamiltonian), C.POINTER(BondChain), C.c_int32,
                                       C.POINTER(SweepOpts), C.POINTER(vp)]
        L.su2_sweep_run.argtypes = [vp, vp, C.c_int32, vp, vp, vp, vp]
        L.su2_sweep_checkpoint.argtypes = [vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                           C.POINTER(C.c_int64), vp, vp, vp]
        L.su2_sweep_destroy.argtypes = [vp]
        for name in SYMBOLS:
            if name != "su2_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class Su2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"su2dmrg error {code}: {msg}")
        self.code = code


def _ptr(x):
    """Device/host address of a torch tensor, numpy array or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


def _vec(ctx, x, n, where):
    """Address of a length-n FP64 vector after checking it: a torch tensor or
    numpy array must be float64, contiguous, hold at least n elements and
    live on the context's GPU (where="device") or in host memory
    (where="host"); anything else raises Su2Error(SU2_EINVAL) before the
    library is called.  A plain int is passed through as a raw address (the
    caller vouches for it)."""
    if isinstance(x, int):
        return x
    def bad(msg):
        return Su2Error(SU2_EINVAL, f"{msg} (a {where} vector of {n} float64 is expected)")
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if str(x.dtype) != "torch.float64":
            raise bad(f"dtype {x.dtype}")
        if not x.is_contiguous():
            raise bad("tensor not contiguous")
        if x.numel() < n:
            raise bad(f"tensor has {x.numel()} elements")
        if where == "device":
            if not x.is_cuda or x.device.index != ctx.device:
                raise bad(f"tensor on {x.device}, the context is on cuda:{ctx.device}")
        elif x.is_cuda:
            raise bad("tensor on a GPU")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if where != "host":
            raise bad("numpy array given for device memory")
        if x.dtype != np.float64:
            raise bad(f"dtype {x.dtype}")
        if not x.flags.c_contiguous:
            raise bad("array not contiguous")
        if x.size < n:
            raise bad(f"array has {x.size} elements")
        return x.ctypes.data
    raise TypeError(type(x))


class Context:
    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = lib().su2_ctx_create(device, s, C.byref(h))
        if rc:
            raise Su2Error(rc, "su2_ctx_create failed")
        self.h = h
        self.device = device

    def check(self, rc):
        if rc:
            raise Su2Error(rc, lib().su2_last_error(self.h).decode())

    def status(self):
        """Synchronise and return (then clear) the device status word."""
        v = C.c_int32()
        self.check(lib().su2_ctx_status(self.h, C.byref(v)))
        return v.value

    def wait(self, timeout_s=-1.0):
        """su2_ctx_wait: host watchdog on the context stream; returns the
        status code (SU2_OK, SU2_ETIMEOUT) instead of raising for a timeout."""
        rc = lib().su2_ctx_wait(self.h, float(timeout_s))
        if rc not in (SU2_OK, SU2_ETIMEOUT):
            self.check(rc)
        return rc

    def close(self):
        if self.h:
            lib().su2_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _sector_array(secs):
    arr = (Sector * max(1, len(secs)))()
    for i, (N, s, d) in enumerate(secs):
        arr[i] = Sector(N, s, d)
    return arr


class Sectors:
    """su2_build_sectors: psi blocks of a two-site window."""

    def __init__(self, ctx: Context, left, right, site_kind, N, twoS):
        self.ctx = ctx
        h = C.c_void_p()
        la, ra = _sector_array(left), _sector_array(right)
        ctx.check(lib().su2_build_sectors(ctx.h, la, len(left), ra, len(right), site_kind, N, twoS,
                                          C.byref(h)))
        self.h = h
        n = C.c_int64()
        nb = C.c_int32()
        bp = C.POINTER(Block)()
        ctx.check(lib().su2_sectors_query(h, C.byref(n), C.byref(nb), C.byref(bp)))
        self.psi_len = n.value
        self.blocks = [(bp[i].a, bp[i].s1, bp[i].s2, bp[i].b, bp[i].jL1, bp[i].j2R, bp[i].rows,
                        bp[i].cols, bp[i].offset) for i in range(nb.value)]
        self.left, self.right = list(left), list(right)

    def close(self):
        if self.h:
            lib().su2_sectors_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _chain(chain):
    offs = [0]
    flat = []
    for bond in chain:
        flat.extend(bond)
        offs.append(len(flat))
    oarr = (C.c_int32 * len(offs))(*offs)
    sarr = _sector_array(flat)
    ch = BondChain(len(chain), C.cast(oarr, C.POINTER(C.c_int32)), C.cast(sarr, C.POINTER(Sector)))
    return ch, (oarr, sarr)


class Environment:
    """su2_build_environment: operator-table, block operators, C~ table, tasks."""

    def __init__(self, ctx: Context, sectors: Sectors, model, left_chain, right_chain, n_left=0, n_right=0,
                 J=1.0, seed=0, t_budget_bytes=0, n_slices=0, prepare_split=False, autotune=False,
                 split_tol=0.0, shard=(0, 0), spin_limit=0, h=None, eri=None, resident_bytes=0,
                 mps_left=None, mps_right=None):
        self.ctx = ctx
        if model == SU2_MODEL_AB_INITIO:
            L = n_left + 2 + n_right
            if h is None or eri is None:
                raise Su2Error(SU2_EINVAL, "the ab initio model needs the integrals h and eri")
            h = np.ascontiguousarray(h, dtype=np.float64)
            eri = np.ascontiguousarray(eri, dtype=np.float64)
            if h.shape != (L, L) or eri.shape != (L, L, L, L):
                raise Su2Error(SU2_EINVAL, f"integrals must be ({L}, {L}) and ({L},)*4 arrays")
        ml, mr = _mps(mps_left), _mps(mps_right)
        H = Hamiltonian(model, n_left, n_right, J, seed, None if h is None else h.ctypes.data,
                        None if eri is None else eri.ctypes.data, None if ml is None else ml.ctypes.data,
                        None if mr is None else mr.ctypes.data)
        lc, keep1 = _chain(left_chain)
        rc_, keep2 = _chain(right_chain)
        opts = EnvOpts(t_budget_bytes, n_slices, 1 if prepare_split else 0, 1 if autotune else 0, split_tol,
                       shard[0], shard[1], spin_limit, int(resident_bytes))
        h = C.c_void_p()
        ctx.check(lib().su2_build_environment(ctx.h, C.byref(H), C.byref(lc), C.byref(rc_), sectors.h,
                                              C.byref(opts), C.byref(h)))
        self.h = h
        info = EnvInfo()
        ctx.check(lib().su2_env_query(h, C.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in EnvInfo._fields_}
        self.psi_len = info.psi_len

    def tasks(self):
        n = self.info["n_tasks"]
        rows = np.zeros((n, 8), dtype=np.int32)
        v = np.zeros(n, dtype=np.float64)
        self.ctx.check(lib().su2_env_tasks(self.h, rows.ctypes.data, v.ctypes.data, n))
        return rows, v

    def terms(self):
        """(left op id, right op id, k, alpha) per operator-table row."""
        n = self.info["n_terms"]
        a = np.zeros(n, dtype=np.int32)
        d = np.zeros(n, dtype=np.int32)
        k = np.zeros(n, dtype=np.int32)
        al = np.zeros(n, dtype=np.float64)
        self.ctx.check(lib().su2_env_terms(self.h, a.ctypes.data, d.ctypes.data, k.ctypes.data, al.ctypes.data, n))
        return a, d, k, al

    def operator_block(self, side, op, qo, qi, rows, cols):
        out = np.zeros((cols, rows), dtype=np.float64)
        self.ctx.check(lib().su2_env_operator_block(self.h, side, op, qo, qi, out.ctypes.data, rows, cols))
        return out.T

    def profile(self, on=True):
        self.ctx.check(lib().su2_profile_enable(self.h, 1 if on else 0))

    def profile_reset(self):
        self.ctx.check(lib().su2_profile_reset(self.h))

    def profile_read(self):
        """{name: (launches, ms, flops)} per kernel kind."""
        out = {}
        for kind in range(6):
            n, ms, fl, nm = C.c_int64(), C.c_double(), C.c_double(), C.c_char_p()
            self.ctx.check(lib().su2_profile_read(self.h, kind, C.byref(n), C.byref(ms), C.byref(fl),
                                                  C.byref(nm)))
            out[nm.value.decode()] = (n.value, ms.value, fl.value)
        return out

    def close(self):
        if self.h:
            lib().su2_env_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_heff(ctx: Context, env: Environment, psi_in, psi_out, prec=SU2_FP64):
    n = env.psi_len
    ctx.check(lib().su2_apply_heff(ctx.h, env.h, _vec(ctx, psi_in, n, "device"), _vec(ctx, psi_out, n, "device"),
                                   prec))


def apply_heff_host(ctx: Context, env: Environment, psi_in, psi_out, prec=SU2_FP64):
    n = env.psi_len
    ctx.check(lib().su2_apply_heff_host(ctx.h, env.h, _vec(ctx, psi_in, n, "host"), _vec(ctx, psi_out, n, "host"),
                                        prec))


def apply_heff_static_scratch(ctx: Context, env: Environment, psi_in, psi_out):
    """su2_apply_heff_static_scratch: FP64 H.psi that allocates nothing
    (its intermediate lives in a fixed 64 MiB device array)."""
    n = env.psi_len
    ctx.check(lib().su2_apply_heff_static_scratch(ctx.h, env.h, _vec(ctx, psi_in, n, "device"),
                                                  _vec(ctx, psi_out, n, "device")))


def diag_heff(ctx: Context, env: Environment, diag_out):
    ctx.check(lib().su2_diag_heff(ctx.h, env.h, _vec(ctx, diag_out, env.psi_len, "device")))


class Davidson:
    """su2_davidson_create / su2_davidson_step / su2_energy."""

    def __init__(self, ctx: Context, env: Environment, psi0, tol=1e-8, max_sub=24, keep=2, max_iter=200,
                 prec=SU2_FP64, use_graph=False):
        self.ctx = ctx
        h = C.c_void_p()
        o = DavOpts(tol, max_sub, keep, max_iter, prec, 1 if use_graph else 0)
        ctx.check(lib().su2_davidson_create(ctx.h, env.h, _vec(ctx, psi0, env.psi_len, "device"), C.byref(o),
                                            C.byref(h)))
        self.h = h
        self.n = env.psi_len
        self.env = env  # the solver reads the environment: keep it alive as long as the solver

    def step(self):
        th, r = C.c_double(), C.c_double()
        self.ctx.check(lib().su2_davidson_step(self.ctx.h, self.h, C.byref(th), C.byref(r)))
        return th.value, r.value

    def solve(self):
        th, r, it = C.c_double(), C.c_double(), C.c_int32()
        rc = lib().su2_davidson_solve(self.ctx.h, self.h, C.byref(th), C.byref(r), C.byref(it))
        if rc not in (SU2_OK, SU2_ENOTCONV):
            self.ctx.check(rc)
        return th.value, r.value, it.value, rc == SU2_OK

    def energy(self):
        e = C.c_double()
        self.ctx.check(lib().su2_energy(self.h, C.byref(e)))
        return e.value

    def energy_check(self, prec=SU2_FP64):
        """(<x|Hx>/<x|x>, ||Hx - rq x||/||x||) of the current Ritz vector x,
        H.x recomputed on the path `prec` (su2_energy_check)."""
        rq, res = C.c_double(), C.c_double()
        self.ctx.check(lib().su2_energy_check(self.ctx.h, self.h, prec, C.byref(rq), C.byref(res)))
        return rq.value, res.value

    def vector(self, out):
        self.ctx.check(lib().su2_davidson_vector(self.ctx.h, self.h, _vec(self.ctx, out, self.n, "device")))

    def close(self):
        if self.h:
            lib().su2_davidson_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sweep:
    """su2_sweep_create / su2_sweep_run: the two-site sweep (target spin
    twoS / 2) on the GPU, of the ab initio model of the integrals (h, eri)
    or, with h = eri = None, of the spin-1/2 Heisenberg chain of
    len(right_chain) + 1 sites with coupling J; it starts at window 0 moving right with the right blocks of
    `right_chain` (bonds of 0 .. L-2 sites) grown by the seeded MPS tensors,
    or by the caller's (`mps_right`, the layout of su2_hamiltonian)."""

    def __init__(self, ctx: Context, h, eri, right_chain, N, D, prec=SU2_SPLIT_BF16, tol=1e-8, max_iter=400,
                 n_slices=5, seed=0, guess_seed=1, mps_right=None, predict=False, J=1.0, twoS=0):
        self.ctx = ctx
        mr = _mps(mps_right)
        if h is None and eri is None:
            L = len(right_chain) + 1
            self._keep = (mr,)
            H = Hamiltonian(SU2_MODEL_HEISENBERG, 0, L - 2, J, seed, None, None, None,
                            None if mr is None else mr.ctypes.data)
        else:
            h = np.ascontiguousarray(h, dtype=np.float64)
            eri = np.ascontiguousarray(eri, dtype=np.float64)
            L = h.shape[0]
            if eri.shape != (L, L, L, L) or len(right_chain) != L - 1:
                raise Su2Error(SU2_EINVAL, "integrals or chain of the wrong size")
            self._keep = (h, eri, mr)
            H = Hamiltonian(SU2_MODEL_AB_INITIO, 0, L - 2, 1.0, seed, h.ctypes.data, eri.ctypes.data, None,
                            None if mr is None else mr.ctypes.data)
        rc_, keep = _chain(right_chain)
        o = SweepOpts(D, prec, tol, max_iter, n_slices, guess_seed, 1 if predict else 0, twoS)
        hd = C.c_void_p()
        ctx.check(lib().su2_sweep_create(ctx.h, C.byref(H), C.byref(rc_), N, C.byref(o), C.byref(hd)))
        self.h = hd
        self.L = L

    def run(self, n_steps, stats=False):
        """(energies, discarded weights) of the next n_steps windows; with
        `stats` also their Davidson iterations and the Rayleigh quotients of
        their start vectors."""
        e = np.zeros(n_steps)
        w = np.zeros(n_steps)
        it = np.zeros(n_steps, dtype=np.int32)
        e0 = np.zeros(n_steps)
        self.ctx.check(lib().su2_sweep_run(self.ctx.h, self.h, n_steps, e.ctypes.data, w.ctypes.data,
                                           it.ctypes.data, e0.ctypes.data))
        return (e, w, it, e0) if stats else (e, w)

    def checkpoint(self):
        """(right chain, MPS tensors) at the start of a right-moving
        half-sweep (su2_sweep_checkpoint): Sweep(..., right_chain=chain,
        mps_right=tensors) continues from there."""
        nb, ns, nv = C.c_int32(), C.c_int32(), C.c_int64()
        self.ctx.check(lib().su2_sweep_checkpoint(self.ctx.h, self.h, C.byref(nb), C.byref(ns), C.byref(nv),
                                                  None, None, None))
        off = np.zeros(nb.value + 1, dtype=np.int32)
        sec = (Sector * max(1, ns.value))()
        mps = np.zeros(max(1, nv.value))
        self.ctx.check(lib().su2_sweep_checkpoint(self.ctx.h, self.h, C.byref(nb), C.byref(ns), C.byref(nv),
                                                  off.ctypes.data, C.cast(sec, C.c_void_p), mps.ctypes.data))
        chain = [[(sec[i].N, sec[i].twoS, sec[i].dim) for i in range(off[k], off[k + 1])] for k in range(nb.value)]
        return chain, mps[:nv.value].copy()

    def close(self):
        if self.h:
            lib().su2_sweep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hash_group(worker, workers, group_count, i):
    """su2_hash_group: the group worker `worker` of `workers` picks at its
    i-th pick (Fig. 2 order)."""
    g = C.c_int64()
    rc = lib().su2_hash_group(worker, workers, group_count, i, C.byref(g))
    if rc:
        raise Su2Error(rc, "su2_hash_group: invalid arguments")
    return g.value


# same names as the C-ABI entry points
build_sectors = Sectors
build_environment = Environment
davidson_create = Davidson


def davidson_step(dav: Davidson):
    return dav.step()


def energy(dav: Davidson):
    return dav.energy()
