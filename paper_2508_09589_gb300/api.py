"""Python binding over the C ABI (argument marshalling only; every step runs in libst.so).

Host inputs are numpy arrays; device inputs are CUDA torch tensors, passed by
pointer.  Calls that hand device pointers to the library first synchronise the
current torch stream, and the library synchronises its own stream before it
returns from a component call, so no ordering hazard crosses the boundary.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, Optional, Sequence

import numpy as np

from . import _lib as L


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _sync_torch(x=None):
    if x is None or _is_torch(x):
        try:
            import torch
            if torch.cuda.is_available():
                torch.cuda.current_stream().synchronize()
        except ImportError:
            pass


def _material(m: Optional[dict]) -> L.Material:
    d = dict(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)
    if m:
        d.update(m)
    return L.Material(float(d["C_ins"]), float(d["C_con"]), float(d["k_ins"]), float(d["k_con"]),
                      int(d["p_c"]), int(d["p_k"]))


def mesh_desc(ns: Sequence[int], nt: int, *, ext: Optional[Sequence[float]] = None, tau: float = 1.0,
              material: Optional[dict] = None, bc: str = "patch_left", bc_width: float = 0.1,
              lambda_crit: float = 0.5, coarse_dof_cap: int = 2000, max_levels: int = 0,
              coarsening: str = "semi", device: int = 0, coarse_solver: str = "auto",
              coarse_max_it: int = 0, coarse_rtol: float = 0.0, march_blocks: int = 0,
              smoother: str = "gmres", smoother_omega: float = 0.5) -> L.MeshDesc:
    d = L.MeshDesc()
    L.lib().st_mesh_desc_default(C.byref(d))
    d.ndim_space = len(ns)
    for q, v in enumerate(ns):
        d.n[q] = int(v)
    d.n_t = int(nt)
    ext = list(ext) if ext else [1.0] * len(ns)
    for q, v in enumerate(ext):
        d.ext[q] = float(v)
    d.tau = float(tau)
    d.mat = _material(material)
    d.bc = L.BC[bc]
    d.bc_width = float(bc_width)
    d.lambda_crit = float(lambda_crit)
    d.coarse_dof_cap = int(coarse_dof_cap)
    d.max_levels = int(max_levels)
    d.coarsening = L.COARSEN[coarsening]
    d.device = int(device)
    d.coarse_solver = L.COARSE[coarse_solver]
    d.coarse_max_it = int(coarse_max_it)
    d.coarse_rtol = float(coarse_rtol)
    d.march_blocks = int(march_blocks)
    d.smoother = L.SMOOTHER[smoother]
    d.smoother_omega = float(smoother_omega)
    return d


def options(rtol: float = 1e-8, max_it: int = 200, restart: int = 30, precision: str = "mixed",
            warm_start: bool = False, smooth_steps: int = 10, use_graphs: bool = True) -> L.Options:
    o = L.Options()
    L.lib().st_options_default(C.byref(o))
    o.rtol = float(rtol)
    o.max_it = int(max_it)
    o.restart = int(restart)
    o.precision = L.PREC[precision]
    o.warm_start = int(bool(warm_start))
    o.smooth_steps = int(smooth_steps)
    o.use_graphs = int(bool(use_graphs))
    return o


def source(kind: str = "uniform", q0: float = 1.0, a: float = 1.0, b: float = 0.5, f: float = 4.0) -> L.Source:
    return L.Source(L.SRC[kind], float(q0), float(a), float(b), float(f))


class Mesh:
    """One space-time problem on one GPU (st_create_mesh ... st_destroy_mesh)."""

    def __init__(self, ns: Sequence[int], nt: int, **kw):
        self.desc = mesh_desc(ns, nt, **kw)
        self.ns = tuple(int(v) for v in ns)
        self.nt = int(nt)
        h = C.c_void_p()
        L.check(L.lib().st_create_mesh(C.byref(self.desc), C.byref(h)), "st_create_mesh")
        self._h = h
        info = L.MeshInfo()
        L.check(L.lib().st_mesh_info_get(self._h, C.byref(info)), "st_mesh_info_get")
        self.n_levels = info.n_levels
        self.n_nodes = info.n_nodes
        self.n_elem = info.n_elem
        self.layout = None

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            L.lib().st_destroy_mesh(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- info
    @property
    def node_shape(self):
        return (self.nt + 1,) + tuple(n + 1 for n in reversed(self.ns))

    @property
    def device_bytes(self) -> int:
        info = L.MeshInfo()
        L.check(L.lib().st_mesh_info_get(self._h, C.byref(info)), "st_mesh_info_get")
        return info.device_bytes

    def levels(self):
        out = []
        for l in range(self.n_levels):
            li = L.LevelInfo()
            L.check(L.lib().st_level_info_get(self._h, l, C.byref(li)), "st_level_info_get")
            sd = len(self.ns)
            out.append(dict(ns=tuple(li.n[q] for q in range(sd)), nt=li.n_t, n_nodes=li.n_nodes,
                            to_next={0: "space", 1: "time", 2: "full", -1: ""}[li.to_next],
                            h=tuple(li.h[q] for q in range(sd)), dt=li.dt))
        return out

    def set_stream(self, stream_ptr: int = 0):
        L.check(L.lib().st_set_stream(self._h, C.c_void_p(stream_ptr)), "st_set_stream")

    def synchronize(self):
        L.check(L.lib().st_synchronize(self._h), "st_synchronize")

    # -- design and solves
    def set_design(self, gamma, layout: Optional[str] = None):
        sp = int(np.prod(self.ns))
        if _is_torch(gamma):
            assert gamma.is_cuda and gamma.dtype.__repr__().endswith("float64") and gamma.is_contiguous()
            n = gamma.numel()
            ptr, mem = gamma.data_ptr(), L.MEM_DEVICE
            _sync_torch(gamma)
        else:
            arr = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
            n = arr.size
            self._gkeep = arr
            ptr, mem = arr.ctypes.data, L.MEM_HOST
        if layout is None:
            layout = "extruded" if n == sp else "spacetime"
        L.check(L.lib().st_set_design(self._h, C.c_void_p(ptr), L.LAYOUT[layout], n, mem), "st_set_design")
        self.layout = layout
        self.design_size = n

    def solve_forward(self, src: Optional[L.Source] = None, opts: Optional[L.Options] = None,
                      allow_not_converged: bool = False, **kw) -> Dict:
        src = src or source(**{k: v for k, v in kw.items() if k in ("kind", "q0", "a", "b", "f")})
        opts = opts or options(**{k: v for k, v in kw.items() if k not in ("kind", "q0", "a", "b", "f")})
        st = L.Stats()
        code = L.lib().st_solve_forward(self._h, C.byref(src), C.byref(opts), C.byref(st))
        L.check(code, "st_solve_forward", allow=(-3,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = code
        return d

    def solve_adjoint(self, objective: str = "compliance", P: int = 20, opts: Optional[L.Options] = None,
                      allow_not_converged: bool = False, **kw):
        obj = L.Objective(L.OBJ[objective], int(P))
        opts = opts or options(**kw)
        st = L.Stats()
        phi = C.c_double()
        code = L.lib().st_solve_adjoint(self._h, C.byref(obj), C.byref(opts), C.byref(phi), C.byref(st))
        L.check(code, "st_solve_adjoint", allow=(-3,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = code
        return phi.value, d

    def sensitivities(self, out=None):
        n = self.design_size
        if out is not None and _is_torch(out):
            _sync_torch(out)
            L.check(L.lib().st_sensitivities(self._h, C.c_void_p(out.data_ptr()), n, L.MEM_DEVICE),
                    "st_sensitivities")
            return out
        arr = np.empty(n, dtype=np.float64)
        L.check(L.lib().st_sensitivities(self._h, C.c_void_p(arr.ctypes.data), n, L.MEM_HOST), "st_sensitivities")
        return arr

    def state(self, which: str = "T", out=None):
        n = self.n_nodes
        if out is not None and _is_torch(out):
            _sync_torch(out)
            L.check(L.lib().st_get_state(self._h, L.WHICH[which], C.c_void_p(out.data_ptr()), n, L.MEM_DEVICE),
                    "st_get_state")
            return out
        arr = np.empty(n, dtype=np.float64)
        L.check(L.lib().st_get_state(self._h, L.WHICH[which], C.c_void_p(arr.ctypes.data), n, L.MEM_HOST),
                "st_get_state")
        return arr

    def set_state(self, s):
        arr = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
        L.check(L.lib().st_set_state(self._h, C.c_void_p(arr.ctypes.data), arr.size, L.MEM_HOST), "st_set_state")

    # -- component entry points (device tensors)
    def _p(self, t):
        assert _is_torch(t) and t.is_cuda and t.is_contiguous()
        return C.c_void_p(t.data_ptr())

    def apply(self, level: int, x, y, precision: str = "fp64", transpose: bool = False):
        _sync_torch()
        L.check(L.lib().st_op_apply(self._h, level, L.PREC[precision], int(transpose), self._p(x), self._p(y)),
                "st_op_apply")
        return y

    def diag(self, level: int, d, precision: str = "fp64"):
        _sync_torch()
        L.check(L.lib().st_op_diag(self._h, level, L.PREC[precision], self._p(d)), "st_op_diag")
        return d

    def restrict(self, level: int, rf, rc, precision: str = "fp64"):
        _sync_torch()
        L.check(L.lib().st_restrict(self._h, level, L.PREC[precision], self._p(rf), self._p(rc)), "st_restrict")
        return rc

    def prolong(self, level: int, xc, xf, precision: str = "fp64"):
        _sync_torch()
        L.check(L.lib().st_prolong(self._h, level, L.PREC[precision], self._p(xc), self._p(xf)), "st_prolong")
        return xf

    def smooth(self, level: int, b, x, steps: int = 10, zero_init: bool = False, precision: str = "fp64",
               transpose: bool = False):
        _sync_torch()
        L.check(L.lib().st_smooth(self._h, level, L.PREC[precision], int(transpose), self._p(b), self._p(x),
                                  int(steps), int(zero_init)), "st_smooth")
        return x

    def vcycle(self, b, x, precision: str = "fp64", transpose: bool = False):
        _sync_torch()
        L.check(L.lib().st_vcycle(self._h, L.PREC[precision], int(transpose), self._p(b), self._p(x)), "st_vcycle")
        return x

    def level_elements(self, level: int) -> np.ndarray:
        lv = self.levels()[level]
        sd = len(self.ns)
        nsym = (2 ** sd) * (2 ** sd + 1) // 2
        sp = int(np.prod(lv["ns"]))
        nstore = 2 * sp if self.layout == "extruded" else sp * lv["nt"]
        out = np.empty(nstore * 4 * nsym, dtype=np.float64)
        L.check(L.lib().st_level_elements(self._h, level, C.c_void_p(out.ctypes.data), out.size),
                "st_level_elements")
        return out.reshape(nstore, 4, nsym)

    def coarse_inverse(self) -> np.ndarray:
        n = self.levels()[-1]["n_nodes"]
        out = np.empty(n * n, dtype=np.float64)
        L.check(L.lib().st_coarse_inverse(self._h, C.c_void_p(out.ctypes.data), out.size), "st_coarse_inverse")
        return out.reshape(n, n)

    # -- design filter and projection (Sec. 3.3.2)
    def filter(self, gamma, r_x: float = 0.0, r_t: float = 0.0, rtol: float = 1e-12, max_it: int = 2000, out=None):
        """PDE-filtered element field (st_filter); numpy in -> numpy out, CUDA tensor in -> tensor out.
        Returns (field, CG iterations)."""
        its = C.c_int()
        if _is_torch(gamma):
            import torch
            out = out if out is not None else torch.empty_like(gamma)
            _sync_torch(gamma)
            L.check(L.lib().st_filter(self._h, C.c_void_p(gamma.data_ptr()), C.c_void_p(out.data_ptr()), gamma.numel(),
                                      L.MEM_DEVICE, float(r_x), float(r_t), float(rtol), int(max_it), C.byref(its)),
                    "st_filter")
            return out, its.value
        arr = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
        res = np.empty_like(arr)
        L.check(L.lib().st_filter(self._h, C.c_void_p(arr.ctypes.data), C.c_void_p(res.ctypes.data), arr.size,
                                  L.MEM_HOST, float(r_x), float(r_t), float(rtol), int(max_it), C.byref(its)),
                "st_filter")
        return res, its.value

    def heaviside(self, x, beta: float = 32.0, eta: float = 0.5):
        """(H(x), H'(x)) of the projection (st_heaviside), host arrays."""
        arr = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        h = np.empty_like(arr)
        dh = np.empty_like(arr)
        L.check(L.lib().st_heaviside(self._h, C.c_void_p(arr.ctypes.data), C.c_void_p(h.ctypes.data),
                                     C.c_void_p(dh.ctypes.data), arr.size, L.MEM_HOST, float(beta), float(eta)),
                "st_heaviside")
        return h, dh

    def apply_timer(self, enable: bool = True):
        """Start (reset) or stop CUDA-event timing of the level-0 smoother operator apply."""
        L.check(L.lib().st_apply_timer(self._h, int(bool(enable))), "st_apply_timer")

    def apply_timer_read(self):
        """(summed launch time in ms, number of timed launches) since apply_timer(True)."""
        ms = C.c_double()
        n = C.c_longlong()
        L.check(L.lib().st_apply_timer_read(self._h, C.byref(ms), C.byref(n)), "st_apply_timer_read")
        return ms.value, n.value


def _batch_args(meshes):
    n = len(meshes)
    arr = (C.c_void_p * n)(*[m._h.value for m in meshes])
    return n, arr


def solve_forward_batch(meshes, src: Optional[L.Source] = None, opts: Optional[L.Options] = None,
                        allow_not_converged: bool = False, sources=None, **kw):
    """Forward solves of several meshes together (st_solve_forward_batch): shared graph
    launches, outer iterations and convergence tests on the device.  Returns per-mesh stats
    dicts (with "status")."""
    n, arr = _batch_args(meshes)
    if sources is None:
        one = src or source(**{k: v for k, v in kw.items() if k in ("kind", "q0", "a", "b", "f")})
        sources = [one] * n
    srcs = (L.Source * n)(*sources)
    opts = opts or options(**{k: v for k, v in kw.items() if k not in ("kind", "q0", "a", "b", "f")})
    st = (L.Stats * n)()
    status = (C.c_int * n)()
    code = L.lib().st_solve_forward_batch(C.cast(arr, C.c_void_p), n, C.cast(srcs, C.c_void_p), C.byref(opts),
                                         C.cast(st, C.c_void_p), C.cast(status, C.c_void_p))
    L.check(code, "st_solve_forward_batch", allow=(-3,) if allow_not_converged else ())
    return [dict(st[k].as_dict(), status=status[k]) for k in range(n)]


def solve_adjoint_batch(meshes, objective: str = "compliance", P: int = 20, opts: Optional[L.Options] = None,
                        allow_not_converged: bool = False, **kw):
    """Adjoint solves of several meshes together (st_solve_adjoint_batch).  Returns (phi list,
    per-mesh stats dicts)."""
    n, arr = _batch_args(meshes)
    objs = (L.Objective * n)(*[L.Objective(L.OBJ[objective], int(P))] * n)
    opts = opts or options(**kw)
    st = (L.Stats * n)()
    status = (C.c_int * n)()
    phi = (C.c_double * n)()
    code = L.lib().st_solve_adjoint_batch(C.cast(arr, C.c_void_p), n, C.cast(objs, C.c_void_p), C.byref(opts),
                                         C.cast(phi, C.c_void_p), C.cast(st, C.c_void_p),
                                         C.cast(status, C.c_void_p))
    L.check(code, "st_solve_adjoint_batch", allow=(-3,) if allow_not_converged else ())
    return [phi[k] for k in range(n)], [dict(st[k].as_dict(), status=status[k]) for k in range(n)]


def plan_hierarchy(ns, nt, **kw):
    """Algorithm 1 levels for a mesh description (host only, no GPU needed)."""
    d = mesh_desc(ns, nt, **kw)
    arr = (L.LevelInfo * 64)()
    n = C.c_int()
    L.check(L.lib().st_plan_hierarchy(C.byref(d), arr, 64, C.byref(n)), "st_plan_hierarchy")
    sd = len(ns)
    return [dict(ns=tuple(arr[l].n[q] for q in range(sd)), nt=arr[l].n_t, n_nodes=arr[l].n_nodes,
                 to_next={0: "space", 1: "time", 2: "full", -1: ""}[arr[l].to_next]) for l in range(n.value)]


def footprint_bytes(ns, nt, precision: str = "mixed", restart: int = 30, **kw) -> int:
    d = mesh_desc(ns, nt, **kw)
    return int(L.lib().st_footprint_bytes(C.byref(d), L.PREC[precision], int(restart)))


class Server:
    """Continuous-batching request server (st_server_create / st_submit / st_poll)."""

    def __init__(self, hbm_budget: int, max_inflight: int = 4, device: int = 0, max_batch: int = 0,
                 batch_nodes: int = 0):
        d = L.ServerDesc(int(hbm_budget), int(max_inflight), int(device), int(max_batch), int(batch_nodes))
        h = C.c_void_p()
        L.check(L.lib().st_server_create(C.byref(d), C.byref(h)), "st_server_create")
        self._h = h
        self._keep = {}

    def submit(self, ns, nt, gamma, layout: Optional[str] = None, src: Optional[L.Source] = None,
               opts: Optional[L.Options] = None, objective: str = "compliance", P: int = 20,
               want_gradient: bool = True, **mesh_kw) -> int:
        arr = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64)).reshape(-1)
        if layout is None:
            layout = "extruded" if arr.size == int(np.prod(ns)) else "spacetime"
        r = L.Request()
        r.mesh = mesh_desc(ns, nt, **mesh_kw)
        r.gamma = arr.ctypes.data_as(C.POINTER(C.c_double))
        r.layout = L.LAYOUT[layout]
        r.count = arr.size
        r.source = src or source()
        r.objective = L.Objective(L.OBJ[objective], int(P))
        r.options = opts or options()
        r.want_gradient = int(bool(want_gradient))
        t = C.c_uint64()
        L.check(L.lib().st_submit(self._h, C.byref(r), C.byref(t)), "st_submit")
        self._keep[t.value] = arr.size
        return t.value

    def cancel(self, ticket: int) -> int:
        """Cancel a queued request (st_cancel).  Returns 0 when it was removed from the queue
        (its result then carries status ST_ERR_CANCELLED), else the library's status code:
        -7 running, -8 finished, -9 unknown."""
        return int(L.lib().st_cancel(self._h, C.c_uint64(ticket)))

    def poll(self, ticket: int):
        """(done, result dict or None, gradient or None)."""
        res = L.Result()
        done = C.c_int()
        n = self._keep.get(ticket, 0)
        grad = np.empty(n, dtype=np.float64)
        L.check(L.lib().st_poll(self._h, C.c_uint64(ticket), C.byref(res), C.c_void_p(grad.ctypes.data), n,
                                C.byref(done)), "st_poll")
        if not done.value:
            return False, None, None
        self._keep.pop(ticket, None)
        out = dict(status=res.status, phi=res.phi, forward=res.forward.as_dict(), adjoint=res.adjoint.as_dict(),
                   latency_s=res.latency_s, queue_s=res.queue_s, footprint=res.footprint, batch=res.batch)
        return True, out, grad

    def wait(self, ticket: int, timeout: float = 600.0, poll_s: float = 0.001):
        import time
        t0 = time.time()
        while True:
            done, res, grad = self.poll(ticket)
            if done:
                return res, grad
            if time.time() - t0 > timeout:
                raise TimeoutError(f"request {ticket} not finished after {timeout} s")
            time.sleep(poll_s)

    def close(self):
        if getattr(self, "_h", None):
            L.lib().st_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MMA:
    """Method of Moving Asymptotes with one constraint on the device (st_mma_*): the optimiser of
    the topology-optimisation loop (Sec. 3.3.3).  x, df0 and dg1 are CUDA float64 tensors of n
    values; update() replaces x by the next iterate and returns the dual multiplier."""

    def __init__(self, n: int, **params):
        p = L.MmaParams()
        L.lib().st_mma_params_default(C.byref(p))
        for k, v in params.items():
            setattr(p, k, float(v))
        self.n = int(n)
        self.it = 0
        h = C.c_void_p()
        L.check(L.lib().st_mma_create(self.n, C.byref(p), C.byref(h)), "st_mma_create")
        self._h = h

    def update(self, x, df0, g1: float, dg1, xmin: float = 0.0, xmax: float = 1.0) -> float:
        for t in (x, df0, dg1):
            assert _is_torch(t) and t.is_cuda and t.dtype.__repr__().endswith("float64") and t.is_contiguous()
            assert t.numel() == self.n
        _sync_torch(x)
        self.it += 1
        lam = C.c_double()
        L.check(L.lib().st_mma_update(self._h, self.it, C.c_void_p(x.data_ptr()), C.c_void_p(df0.data_ptr()),
                                      float(g1), C.c_void_p(dg1.data_ptr()), float(xmin), float(xmax), None,
                                      C.byref(lam)), "st_mma_update")
        return lam.value

    def close(self):
        if self._h:
            L.lib().st_mma_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TopOpt:
    """The topology-optimisation loop of Sec. 3.3 on a mesh (st_topopt_*): each step() is one
    design iteration (filter, projection, design, forward and adjoint solves, chain rule,
    volume constraint, MMA update), all in the library.  gamma0 is a numpy array or a CUDA
    float64 tensor in the mesh's design layout.  Parameters: vf, r_x, r_t, beta, eta,
    objective ("pnorm" or "compliance"), P, obj_scale, filter_rtol, filter_max_it, warm_start
    and the MMA's (s0, incr, decr, move, raa, lam_max)."""

    def __init__(self, mesh: Mesh, gamma0, layout: Optional[str] = None, **params):
        p = L.TopOptParams()
        L.lib().st_topopt_params_default(C.byref(p))
        for k, v in params.items():
            if k == "objective":
                p.objective = L.OBJ[v]
            elif k in ("P", "filter_max_it", "warm_start"):
                setattr(p, k, int(v))
            elif k in ("s0", "incr", "decr", "move", "raa", "lam_max"):
                setattr(p.mma, k, float(v))
            else:
                if k not in dict(L.TopOptParams._fields_):
                    raise TypeError(f"unknown parameter {k}")
                setattr(p, k, float(v))
        self.mesh = mesh
        sp = int(np.prod(mesh.ns))
        if _is_torch(gamma0):
            assert gamma0.is_cuda and gamma0.dtype.__repr__().endswith("float64") and gamma0.is_contiguous()
            n, ptr, mem = gamma0.numel(), gamma0.data_ptr(), L.MEM_DEVICE
            _sync_torch(gamma0)
        else:
            arr = np.ascontiguousarray(np.asarray(gamma0, dtype=np.float64))
            n, ptr, mem = arr.size, arr.ctypes.data, L.MEM_HOST
        if layout is None:
            layout = "extruded" if n == sp else "spacetime"
        self.layout = layout
        self.n = n
        self.shape = tuple(reversed(mesh.ns)) if layout == "extruded" else (mesh.nt,) + tuple(reversed(mesh.ns))
        h = C.c_void_p()
        L.check(L.lib().st_topopt_create(mesh._h, C.byref(p), C.c_void_p(ptr), L.LAYOUT[layout], n, mem,
                                         C.byref(h)), "st_topopt_create")
        self._h = h
        mesh.design_size = n
        mesh.layout = layout

    def step(self, src: Optional[L.Source] = None, opts: Optional[L.Options] = None,
             allow_not_converged: bool = False, **kw) -> Dict:
        """One design iteration; returns its statistics (phi, chi, lam, change, solver stats)."""
        src = src or source(**{k: v for k, v in kw.items() if k in ("kind", "q0", "a", "b", "f")})
        opts = opts or options(**{k: v for k, v in kw.items() if k not in ("kind", "q0", "a", "b", "f")})
        st = L.TopOptStats()
        code = L.lib().st_topopt_step(self._h, C.byref(src), C.byref(opts), C.byref(st))
        L.check(code, "st_topopt_step", allow=(-3,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = code
        return d

    def get(self, which: str = "gamma", out=None):
        """A field of the loop (gamma, gamma_tilde, gamma_bar, dphi, dchi): into a CUDA tensor
        `out`, else a new numpy array in the design's shape."""
        if out is not None and _is_torch(out):
            _sync_torch(out)
            L.check(L.lib().st_topopt_get(self._h, L.TO_FIELD[which], C.c_void_p(out.data_ptr()), self.n,
                                          L.MEM_DEVICE), "st_topopt_get")
            return out
        arr = np.empty(self.n, dtype=np.float64)
        L.check(L.lib().st_topopt_get(self._h, L.TO_FIELD[which], C.c_void_p(arr.ctypes.data), self.n, L.MEM_HOST),
                "st_topopt_get")
        return arr.reshape(self.shape)

    def close(self):
        if getattr(self, "_h", None):
            L.lib().st_topopt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BDF1:
    """The paper's time-stepping reference solver (st_bdf1_*, Sec. 4): backward Euler with
    consistent mass on the spatial mesh of the space-time problem (ns, nt, **mesh keywords as
    for Mesh), each step solved by FGMRES with the library's spatial multigrid."""

    def __init__(self, ns: Sequence[int], nt: int, **kw):
        self.desc = mesh_desc(ns, nt, **kw)
        self.ns = tuple(int(v) for v in ns)
        self.nt = int(nt)
        h = C.c_void_p()
        L.check(L.lib().st_bdf1_create(C.byref(self.desc), C.byref(h)), "st_bdf1_create")
        self._h = h

    @property
    def plane_shape(self):
        return tuple(n + 1 for n in reversed(self.ns))

    def set_design(self, gamma, layout: Optional[str] = None):
        sp = int(np.prod(self.ns))
        if _is_torch(gamma):
            assert gamma.is_cuda and gamma.dtype.__repr__().endswith("float64") and gamma.is_contiguous()
            n, ptr, mem = gamma.numel(), gamma.data_ptr(), L.MEM_DEVICE
            _sync_torch(gamma)
        else:
            arr = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
            n, ptr, mem = arr.size, arr.ctypes.data, L.MEM_HOST
        if layout is None:
            layout = "extruded" if n == sp else "spacetime"
        L.check(L.lib().st_bdf1_set_design(self._h, C.c_void_p(ptr), L.LAYOUT[layout], n, mem), "st_bdf1_set_design")
        self._design_size = n

    def forward(self, src: Optional[L.Source] = None, opts: Optional[L.Options] = None, out=None,
                allow_not_converged: bool = False, **kw):
        """Run the steps; returns (trajectory, stats).  The trajectory (nt + 1 planes) goes to the
        CUDA tensor `out` when given, else to a new numpy array."""
        src = src or source(**{k: v for k, v in kw.items() if k in ("kind", "q0", "a", "b", "f")})
        opts = opts or options(**{k: v for k, v in kw.items() if k not in ("kind", "q0", "a", "b", "f")})
        n = (self.nt + 1) * int(np.prod(self.plane_shape))
        st = L.Bdf1Stats()
        if out is not None and _is_torch(out):
            assert out.numel() == n
            _sync_torch(out)
            ptr, mem, res = out.data_ptr(), L.MEM_DEVICE, out
        else:
            res = np.empty((self.nt + 1,) + self.plane_shape, dtype=np.float64)
            ptr, mem = res.ctypes.data, L.MEM_HOST
        code = L.lib().st_bdf1_forward(self._h, C.byref(src), C.byref(opts), C.c_void_p(ptr), n, mem, C.byref(st))
        L.check(code, "st_bdf1_forward", allow=(-3,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = code
        return res, d

    def adjoint(self, P: int = 20, opts: Optional[L.Options] = None, out=None, allow_not_converged: bool = False,
                **kw):
        """The discrete adjoint for the p-norm objective; returns (phi, multipliers, stats), the
        multipliers into the CUDA tensor `out` when given, else a new numpy array."""
        opts = opts or options(**kw)
        n = (self.nt + 1) * int(np.prod(self.plane_shape))
        st = L.Bdf1Stats()
        phi = C.c_double()
        if out is not None and _is_torch(out):
            assert out.numel() == n
            _sync_torch(out)
            ptr, mem, res = out.data_ptr(), L.MEM_DEVICE, out
        else:
            res = np.empty((self.nt + 1,) + self.plane_shape, dtype=np.float64)
            ptr, mem = res.ctypes.data, L.MEM_HOST
        code = L.lib().st_bdf1_adjoint(self._h, int(P), C.byref(opts), C.byref(phi), C.c_void_p(ptr), n, mem,
                                       C.byref(st))
        L.check(code, "st_bdf1_adjoint", allow=(-3,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = code
        return phi.value, res, d

    def sensitivities(self, out=None):
        """d phi / d gamma of the last adjoint, in the design's layout (CUDA tensor `out` or numpy)."""
        n = self._design_size
        if out is not None and _is_torch(out):
            _sync_torch(out)
            L.check(L.lib().st_bdf1_sensitivities(self._h, C.c_void_p(out.data_ptr()), n, L.MEM_DEVICE),
                    "st_bdf1_sensitivities")
            return out
        arr = np.empty(n, dtype=np.float64)
        L.check(L.lib().st_bdf1_sensitivities(self._h, C.c_void_p(arr.ctypes.data), n, L.MEM_HOST),
                "st_bdf1_sensitivities")
        return arr

    def close(self):
        if getattr(self, "_h", None):
            L.lib().st_bdf1_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
