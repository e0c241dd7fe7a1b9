"""Python binding of the C-ABI: torch tensors in, torch tensors out.

Every step runs in the CUDA library; this module only checks shapes, allocates outputs
with torch (device memory and streams are torch's), and marshals pointers.
"""
from __future__ import annotations

import atexit
import ctypes
import sys
import weakref

import torch

from . import _lib as L

PRECISIONS = {"fp64": L.FIRAL_FP64, "fp32": L.FIRAL_FP32, "mixed": L.FIRAL_MIXED_BF16,
              "mixed_fast": L.FIRAL_MIXED_BF16_FAST}


_LIVE_PROBLEMS = weakref.WeakSet()
_LIVE_HANDLES = weakref.WeakSet()


@atexit.register
def _close_all():
    """Release library objects before interpreter teardown (the CUDA runtime may be gone later)."""
    for p in list(_LIVE_PROBLEMS):
        p.close()
    for h in list(_LIVE_HANDLES):
        h.close()


def _dt(t: torch.Tensor) -> int:
    return {torch.float64: L.FIRAL_DT_F64, torch.float32: L.FIRAL_DT_F32,
            torch.bfloat16: L.FIRAL_DT_BF16}[t.dtype]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def vec_dtype(precision: str):
    return torch.float64 if precision == "fp64" else torch.float32


class Handle:
    """A library handle bound to the current device and torch's current stream."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        self.lib = L.load()
        st = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        L.check(self.lib.firal_create(ctypes.byref(self._h), ctypes.c_void_p(st.cuda_stream)))
        _LIVE_HANDLES.add(self)

    @property
    def ptr(self):
        return self._h

    def set_stream(self, stream: torch.cuda.Stream):
        L.check(self.lib.firal_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), self._h)

    def close(self):
        if self._h:
            self.lib.firal_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def set_default_tuning(self, dterm_splits=0, bsum_splits=0, sm_budget=0):
        """Tuning of every problem created on this handle afterwards (batched pools too)."""
        t = L.FiralTuning(int(dterm_splits), int(bsum_splits), int(sm_budget), 0)
        L.check(self.lib.firal_set_default_tuning(self._h, ctypes.byref(t)), self._h)

    # ---- standalone building blocks
    def block_eigvals(self, Sig: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
        c, d, _ = Sig.shape
        Sig = Sig.contiguous().to(torch.float64)
        H = H.contiguous().to(torch.float64)
        out = torch.empty((c, d), dtype=torch.float64, device=Sig.device)
        L.check(self.lib.firal_block_eigvals(self._h, c, d, _ptr(Sig), _ptr(H), _ptr(out)),
                self._h)
        return out

    def nu_bisect(self, mu: torch.Tensor) -> float:
        mu = mu.contiguous().to(torch.float64)
        nu = ctypes.c_double()
        L.check(self.lib.firal_nu_bisect(self._h, _ptr(mu), mu.numel(), ctypes.byref(nu)),
                self._h)
        return nu.value


class _CudaArray:
    """A device buffer owned by the library, seen by torch without a copy."""

    def __init__(self, ptr, count, dtype):
        typestr = {torch.float32: "<f4", torch.float64: "<f8"}[dtype]
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None,
                                         "stream": None}


def _device_view(ptr, count, dtype, device):
    return torch.as_tensor(_CudaArray(ptr, count, dtype), device=device)


def torch_allreduce(group=None):
    """An allreduce over a torch.distributed process group for ``Problem.set_comm``.  With
    NCCL the device tensor is reduced in place on torch's current stream (the library's); with
    gloo it is staged through host memory."""
    import torch.distributed as dist

    def reduce(t, op):
        rop = dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM
        if t.is_cuda and "nccl" not in str(dist.get_backend(group)):
            h = t.cpu()
            dist.all_reduce(h, op=rop, group=group)
            t.copy_(h)
        else:
            dist.all_reduce(t, op=rop, group=group)
    return reduce


def shard_rows(n: int, world: int, rank: int):
    """Contiguous slice [start, stop) of n pool rows held by ``rank`` of ``world`` processes
    (sizes differ by at most one; the first n % world ranks hold one more)."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _pool(X, h):
    return L.FiralPool(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(h.data_ptr()), X.shape[0],
                       X.shape[1], h.shape[1], _dt(X), _dt(h))


def _hess0(Xo, ho, lam):
    if Xo is None or Xo.shape[0] == 0:
        return L.FiralHess0(None, None, 0, lam)
    return L.FiralHess0(ctypes.c_void_p(Xo.data_ptr()), ctypes.c_void_p(ho.data_ptr()),
                        Xo.shape[0], lam)


def _cg(tol=0.1, maxit=100, fixed_iters=0, block=False):
    return L.FiralCGOpts(tol, maxit, fixed_iters, 1 if block else 0, 0)


class Problem:
    """A prepared problem (pool, labelled set, lambda) for one precision."""

    def __init__(self, handle: Handle, X, h, Xo=None, ho=None, lam=1e-3, precision="fp32"):
        self.handle = handle
        self.lib = handle.lib
        self.precision = precision
        self.vdt = vec_dtype(precision)
        for t in (X, h):
            assert t.is_cuda and t.is_contiguous()
        self.n, self.d = X.shape
        self.c = h.shape[1]
        self.D = self.d * self.c
        self.device = X.device
        pool = _pool(X, h)
        h0 = _hess0(Xo, ho, lam)
        self._p = ctypes.c_void_p()
        L.check(self.lib.firal_problem_create(handle.ptr, ctypes.byref(pool), ctypes.byref(h0),
                                              PRECISIONS[precision], ctypes.byref(self._p)),
                handle.ptr)
        _LIVE_PROBLEMS.add(self)

    def close(self):
        if self._p:
            self.lib.firal_problem_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, code):
        L.check(code, self.handle.ptr)

    def _vec(self, t):
        t = t.to(self.device, self.vdt).contiguous()
        return t

    def probes(self, seed: int, t: int, s: int) -> torch.Tensor:
        V = torch.empty((s, self.D), dtype=self.vdt, device=self.device)
        self._chk(self.lib.firal_probes(self._p, seed, t, s, _ptr(V)))
        return V

    def hessian_apply(self, V: torch.Tensor, z: torch.Tensor | None = None, op: int = 0):
        """op 0: Sigma_z V; op 1: H_p V.  V is (s, D) probe-major."""
        V = self._vec(V)
        zz = self._vec(z) if z is not None else None
        out = torch.empty_like(V)
        self._chk(self.lib.firal_hessian_apply(self._p, op, _ptr(zz), _ptr(V), V.shape[0],
                                               _ptr(out)))
        return out

    def precond_blocks(self, z: torch.Tensor | None = None) -> torch.Tensor:
        zz = self._vec(z) if z is not None else None
        out = torch.empty((self.c, self.d, self.d), dtype=torch.float64, device=self.device)
        self._chk(self.lib.firal_precond_blocks(self._p, _ptr(zz), _ptr(out)))
        return out

    def pcg(self, z, B, tol=0.1, maxit=100, fixed_iters=0, check=True, block=False):
        z, B = self._vec(z), self._vec(B)
        s = B.shape[0]
        X = torch.empty_like(B)
        iters = (ctypes.c_int32 * s)()
        relres = (ctypes.c_double * s)()
        cg = _cg(tol, maxit, fixed_iters, block)
        code = self.lib.firal_pcg(self._p, _ptr(z), _ptr(B), s, ctypes.byref(cg), _ptr(X), iters,
                                  relres)
        if check or code not in (0, -4):
            self._chk(code)
        return X, list(iters), list(relres)

    def quad_forms(self, A, B, scale=1.0):
        A, B = self._vec(A), self._vec(B)
        g = torch.empty(self.n, dtype=self.vdt, device=self.device)
        self._chk(self.lib.firal_quad_forms(self._p, _ptr(A), _ptr(B), A.shape[0], scale, _ptr(g)))
        return g

    def md_step(self, z, g, budget, beta0=1.0):
        z = self._vec(z).clone()
        g = self._vec(g)
        self._chk(self.lib.firal_md_step(self._p, _ptr(z), _ptr(g), budget, beta0))
        return z

    def relax_opts(self, s=10, T=20, tol=0.1, maxit=100, fixed_iters=0, beta0=1.0, seed=1,
                   estimator=0, md_tol=0.0, block_cg=False):
        return L.FiralRelaxOpts(s, T, _cg(tol, maxit, fixed_iters, block_cg), beta0, seed,
                                PRECISIONS[self.precision], estimator, md_tol)

    def relax_step(self, opts, t, budget, z, stats=True):
        st = L.FiralStepStats()
        self._chk(self.lib.firal_relax_step(self._p, ctypes.byref(opts), t, budget, _ptr(z),
                                            ctypes.byref(st) if stats else None))
        if not stats:
            return None
        return dict(fhat=st.fhat, gmax=st.gmax, zmax=st.zmax, cg_iters=list(st.cg_iters),
                    cg_relres=list(st.cg_relres))

    def objective_fwd(self, z, seed, t, s, tol=0.1, maxit=100, fixed_iters=0, keep=True):
        z = self._vec(z)
        cg = _cg(tol, maxit, fixed_iters)
        U = torch.empty((s, self.D), dtype=self.vdt, device=self.device) if keep else None
        Y = torch.empty_like(U) if keep else None
        f = ctypes.c_double()
        self._chk(self.lib.firal_objective_fwd(self._p, _ptr(z), seed, t, s, ctypes.byref(cg),
                                               ctypes.byref(f), _ptr(U), _ptr(Y)))
        return f.value, U, Y

    def objective_bwd(self, z, seed, t, s, U=None, Y=None, grad_out=1.0, tol=0.1, maxit=100,
                      fixed_iters=0):
        z = self._vec(z)
        cg = _cg(tol, maxit, fixed_iters)
        g = torch.empty(self.n, dtype=self.vdt, device=self.device)
        self._chk(self.lib.firal_objective_bwd(self._p, _ptr(z), seed, t, s, ctypes.byref(cg),
                                               _ptr(U), _ptr(Y), grad_out, _ptr(g)))
        return g

    def round(self, z, budget, eta=0.0, exclude_selected=True):
        z = self._vec(z)
        sel = torch.empty(budget, dtype=torch.int32, device=self.device)
        o = L.FiralRoundOpts(eta, 1 if exclude_selected else 0, PRECISIONS[self.precision])
        st = L.FiralRoundStats()
        self._chk(self.lib.firal_round_problem(self._p, _ptr(z), budget, ctypes.byref(o),
                                               _ptr(sel), ctypes.byref(st)))
        return sel, dict(nu_last=st.nu_last, score_last=st.score_last)

    def round_sweep(self, z, budget, etas, exclude_selected=True):
        """Round once per eta (Section 5's choice of eta); returns (selections (n_eta x b),
        criteria min_k lambda_min(H_k) per eta, index of the best eta)."""
        z = self._vec(z)
        ne = len(etas)
        sel = torch.empty((ne, budget), dtype=torch.int32, device=self.device)
        e_arr = (ctypes.c_double * ne)(*[float(e) for e in etas])
        crit = (ctypes.c_double * ne)()
        best = ctypes.c_int32()
        o = L.FiralRoundOpts(0.0, 1 if exclude_selected else 0, PRECISIONS[self.precision])
        self._chk(self.lib.firal_round_sweep(self._p, _ptr(z), budget, e_arr, ne,
                                             ctypes.byref(o), _ptr(sel), crit,
                                             ctypes.byref(best)))
        return sel, list(crit), best.value

    # ---- row sharding (the paper's data decomposition over processes, Section 3.3)
    def set_comm(self, rank: int, world: int, allreduce=None):
        """Join a row-sharded group: this problem holds this process's slice of the pool, and
        ``allreduce(tensor, op)`` (in place, op "sum" or "max"; see ``torch_allreduce``) adds
        the partial sums over points across the group.  ``world == 1`` leaves the group."""
        if world > 1 and allreduce is None:
            raise ValueError("a row-sharded problem needs an allreduce")
        dtypes = {L.FIRAL_DT_F32: torch.float32, L.FIRAL_DT_F64: torch.float64}
        device = self.device

        def cb(ptr, count, dtype, op, stream, user):
            try:
                t = _device_view(ptr, int(count), dtypes[dtype], device)
                allreduce(t, "max" if op == L.FIRAL_REDUCE_MAX else "sum")
                return 0
            except Exception as exc:   # reported as FIRAL_ERR_COMM; no exception crosses the ABI
                self.comm_error = exc
                return 1
        self._comm_cb = L.ALLREDUCE_FN(cb) if world > 1 else L.ALLREDUCE_FN()
        comm = L.FiralComm(int(rank), int(world), self._comm_cb, None)
        self._chk(self.lib.firal_problem_set_comm(self._p, ctypes.byref(comm)))

    # ---- launch tuning (see autotune.py)
    def set_tuning(self, dterm_splits=0, bsum_splits=0, sm_budget=0):
        t = L.FiralTuning(int(dterm_splits), int(bsum_splits), int(sm_budget), 0)
        self._chk(self.lib.firal_problem_set_tuning(self._p, ctypes.byref(t)))

    def get_tuning(self):
        """The split counts and SM budget the problem's last launches used."""
        t = L.FiralTuning()
        self._chk(self.lib.firal_problem_get_tuning(self._p, ctypes.byref(t)))
        return dict(dterm_splits=t.dterm_splits, bsum_splits=t.bsum_splits,
                    sm_budget=t.sm_budget)

    # ---- Exact-FIRAL (Algorithm 1) on dense d~ x d~ matrices
    def exact_objective(self, z, grad=True):
        """``(f, g)``: f = Tr(Sigma_z^{-1} H_p) and the exact gradient g (eq. 6, None when
        grad is False)."""
        z = self._vec(z)
        f = ctypes.c_double()
        g = torch.empty(self.n, dtype=self.vdt, device=self.device) if grad else None
        self._chk(self.lib.firal_exact_objective(self._p, _ptr(z), ctypes.byref(f), _ptr(g)))
        return f.value, g

    def exact_relax(self, budget, T, beta0=1.0, z0=None):
        """Exact Relax: ``(z_diamond, f history)``."""
        z = torch.empty(self.n, dtype=self.vdt, device=self.device)
        z0 = self._vec(z0) if z0 is not None else None
        hist = (ctypes.c_double * max(T, 1))()
        self._chk(self.lib.firal_exact_relax(self._p, float(budget), T, float(beta0), _ptr(z0),
                                             _ptr(z), hist))
        return z, list(hist)[:T]

    def exact_round(self, z, budget, eta=0.0, exclude_selected=True):
        """Exact Round: ``(selected (device int32), trace of each pick, nu_t of each pick)``."""
        z = self._vec(z)
        sel = torch.empty(budget, dtype=torch.int32, device=self.device)
        r = (ctypes.c_double * budget)()
        nu = (ctypes.c_double * budget)()
        self._chk(self.lib.firal_exact_round(self._p, _ptr(z), budget, float(eta),
                                             1 if exclude_selected else 0, _ptr(sel), r, nu))
        return sel, list(r), list(nu)


# ---- active learning (the outer loop of Section 5)
def lr_probs(X, W, precision="fp32", handle: Handle | None = None):
    """h = softmax(X W^T) row by row (eq. 1); X (rows x d) and W (c x d) on the device."""
    H = handle or Handle()
    vdt = vec_dtype(precision)
    X = X.contiguous()
    W = W.to(vdt).contiguous()
    h = torch.empty((X.shape[0], W.shape[0]), dtype=vdt, device=X.device)
    L.check(H.lib.firal_lr_probs(H.ptr, _ptr(X), _dt(X), _ptr(W), X.shape[0], X.shape[1],
                                 W.shape[0], PRECISIONS[precision], _ptr(h)), H.ptr)
    return h


def lr_fit(X, y, c, gamma=1.0, precision="fp32", W0=None, max_newton=30, tol=1e-8,
           handle: Handle | None = None):
    """Ridge-regularised multinomial logistic regression by damped Newton-PCG; returns
    ``(W (c x d), newton_steps, final gradient norm)``."""
    H = handle or Handle()
    vdt = vec_dtype(precision)
    X = X.contiguous()
    y = y.to(torch.int32).contiguous()
    W = (torch.zeros((c, X.shape[1]), dtype=vdt, device=X.device) if W0 is None
         else W0.to(vdt).contiguous().clone())
    it, gn = ctypes.c_int32(), ctypes.c_double()
    L.check(H.lib.firal_lr_fit(H.ptr, _ptr(X), _dt(X), _ptr(y), X.shape[0], X.shape[1], c,
                               float(gamma), PRECISIONS[precision], max_newton, float(tol),
                               _ptr(W), ctypes.byref(it), ctypes.byref(gn)), H.ptr)
    return W, it.value, gn.value


def active_learning(X_pool, y_pool, X_lab, y_lab, c, rounds, budget, *, lam=1e-3,
                    lr_gamma=1.0, precision="fp32", s=10, T=20, tol=0.1, maxit=100,
                    fixed_iters=0, beta0=1.0, seed=1, md_tol=0.0, eta=0.0, lr_max_newton=30,
                    lr_tol=1e-8, handle: Handle | None = None):
    """Multi-round active learning on device tensors: returns ``(selected (rounds x budget)
    pool indices, final classifier W (c x d), last f^ of each round's Relax)``."""
    H = handle or Handle()
    X_pool, y_pool = X_pool.contiguous(), y_pool.to(torch.int32).contiguous()
    m = 0 if X_lab is None else X_lab.shape[0]
    if m:
        X_lab = X_lab.to(X_pool.dtype).contiguous()
        y_lab = y_lab.to(torch.int32).contiguous()
    n, d = X_pool.shape
    ro = L.FiralRelaxOpts(s, T, _cg(tol, maxit, fixed_iters), beta0, seed, PRECISIONS[precision],
                          0, md_tol)
    o = L.FiralAlOpts(rounds, budget, lam, lr_gamma, lr_max_newton, 0, lr_tol, ro, eta)
    sel = torch.empty((rounds, budget), dtype=torch.int32, device=X_pool.device)
    W = torch.empty((c, d), dtype=vec_dtype(precision), device=X_pool.device)
    fh = (ctypes.c_double * rounds)()
    L.check(H.lib.firal_active_learning(H.ptr, _ptr(X_pool), _ptr(y_pool), n,
                                        _ptr(X_lab) if m else None, _ptr(y_lab) if m else None,
                                        m, d, c, _dt(X_pool), ctypes.byref(o), _ptr(sel),
                                        _ptr(W), fh), H.ptr)
    return sel, W, list(fh)


def _to_device(t, device, dtype=None, non_blocking=True):
    if t is None:
        return None
    if dtype is not None and t.dtype != dtype:
        t = t.to(dtype)
    return t.to(device, non_blocking=non_blocking).contiguous()


def relax(X, h, Xo=None, ho=None, lam=1e-3, budget=10.0, *, s=10, T=20, tol=0.1, maxit=100,
          fixed_iters=0, beta0=1.0, seed=1, precision="fp32", estimator=0, md_tol=0.0, z0=None,
          handle: Handle | None = None, device="cuda"):
    """Relax solve (Algorithm 2).  Host (CPU, ideally pinned) or device tensors are accepted;
    host inputs are copied to the device inside the call and z is returned on the inputs'
    device.  Returns ``(z, fhat_history)``."""
    host = not X.is_cuda
    dev = torch.device(device) if host else X.device
    Xd, hd = _to_device(X, dev), _to_device(h, dev)
    Xod, hod = _to_device(Xo, dev), _to_device(ho, dev)
    H = handle or Handle()
    vdt = vec_dtype(precision)
    z = torch.empty(Xd.shape[0], dtype=vdt, device=dev)
    z0d = _to_device(z0, dev, vdt) if z0 is not None else None
    opts = L.FiralRelaxOpts(s, T, _cg(tol, maxit, fixed_iters), beta0, seed,
                            PRECISIONS[precision], estimator, md_tol)
    hist = (ctypes.c_double * max(T, 1))()
    st = L.FiralRelaxStats()
    pool = _pool(Xd, hd)
    h0 = _hess0(Xod, hod, lam)
    L.check(H.lib.firal_relax(H.ptr, ctypes.byref(pool), ctypes.byref(h0), budget, _ptr(z0d),
                              ctypes.byref(opts), _ptr(z), hist, ctypes.byref(st)), H.ptr)
    fh = list(hist)[:st.iters_done]
    if host:
        z = z.to("cpu")
    return z, fh


def batched_relax(problems, *, s=8, T=10, tol=0.1, maxit=100, fixed_iters=0, beta0=1.0, seed=1,
                  precision="mixed", estimator=0, handle: Handle | None = None):
    """Relax (Algorithm 2) on many independent pools in one call.  ``problems`` is a list of
    dicts with device tensors X, h, Xo, ho and floats lam, budget.  Returns the list of z."""
    H = handle or Handle()
    n = len(problems)
    pools = (L.FiralPool * n)(*[_pool(p["X"], p["h"]) for p in problems])
    h0s = (L.FiralHess0 * n)(*[_hess0(p.get("Xo"), p.get("ho"), p.get("lam", 1e-3))
                               for p in problems])
    budgets = (ctypes.c_double * n)(*[float(p["budget"]) for p in problems])
    vdt = vec_dtype(precision)
    zs = [torch.empty(p["X"].shape[0], dtype=vdt, device=p["X"].device) for p in problems]
    zptr = (ctypes.c_void_p * n)(*[z.data_ptr() for z in zs])
    opts = L.FiralRelaxOpts(s, T, _cg(tol, maxit, fixed_iters), beta0, seed,
                            PRECISIONS[precision], estimator, 0.0)
    L.check(H.lib.firal_batched_relax(H.ptr, n, pools, h0s, budgets, ctypes.byref(opts), zptr),
            H.ptr)
    return zs


def round_select(X, h, z, budget, Xo=None, ho=None, lam=1e-3, *, eta=0.0, precision="fp32",
                 handle: Handle | None = None, device="cuda"):
    """Round step (Algorithm 3): returns the selected pool indices (int32, selection order)."""
    host = not X.is_cuda
    dev = torch.device(device) if host else X.device
    Xd, hd = _to_device(X, dev), _to_device(h, dev)
    Xod, hod = _to_device(Xo, dev), _to_device(ho, dev)
    H = handle or Handle()
    zd = _to_device(z, dev, vec_dtype(precision))
    sel = torch.empty(budget, dtype=torch.int32, device=dev)
    o = L.FiralRoundOpts(eta, 1, PRECISIONS[precision])
    st = L.FiralRoundStats()
    pool = _pool(Xd, hd)
    h0 = _hess0(Xod, hod, lam)
    L.check(H.lib.firal_round(H.ptr, ctypes.byref(pool), ctypes.byref(h0), _ptr(zd), budget,
                              ctypes.byref(o), _ptr(sel), ctypes.byref(st)), H.ptr)
    return (sel.to("cpu") if host else sel), dict(nu_last=st.nu_last, score_last=st.score_last)
