"""Thin Python binding of the C ABI in include/fcsdnn.h (ctypes; marshalling only).

Every step of the operator runs in the CUDA library; this module only packs
descriptors, loads the method data files (FC-Gram tables, classifier weights),
and passes device pointers of torch tensors and the current CUDA stream. It
raises if the library is missing: there is no CPU path.
"""
import ctypes as C
import functools
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "_lib", "libfcsdnn.so")
_lib = None

FC_OK = 0
FC_ERR_INVALID, FC_ERR_CUDA, FC_ERR_DONOR, FC_ERR_OVERLAP, FC_ERR_NONFINITE = 1, 2, 3, 4, 5
STATUS = {0: "FC_OK", 1: "FC_ERR_INVALID", 2: "FC_ERR_CUDA", 3: "FC_ERR_DONOR", 4: "FC_ERR_OVERLAP",
          5: "FC_ERR_NONFINITE", 6: "FC_ERR_TIMEOUT", 7: "FC_ERR_UNIMPLEMENTED", 8: "FC_ERR_OOM"}
STEP_FILTER, STEP_FROZEN_MU, STEP_PER_PATCH, STEP_FIXED_DT, STEP_GRAPH = 1, 2, 4, 8, 16
TUNE_PLANS, TUNE_WARPS = 1, 2

# every symbol include/fcsdnn.h declares
EXPORTS = ["fc_init_patches", "fc_state_size", "fc_patch_offset", "fc_active_points", "fc_rhs", "fc_viscosity",
           "fc_filter", "fc_project", "fc_timestep", "fc_rk_step", "fc_rk_step_host", "fc_autotune", "fc_adjoint_step",
           "fc_initial_sensitivity", "fc_drag", "fc_sync_status", "fc_partition", "fc_shard", "fc_shard_counts",
           "fc_launch_count", "fc_profile_enable", "fc_profile_read", "fc_profile_get", "fc_profile_reset",
           "fc_pass_stats", "fc_line_stats", "fc_probe_fp64", "fc_rhs_patch_noalloc", "fc_last_error", "fc_destroy"]


class FcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PatchDescC(C.Structure):
    _fields_ = [("kind", C.c_int), ("n1", C.c_int), ("n2", C.c_int), ("geom", C.c_double * 4),
                ("side", C.c_int * 4), ("bc", (C.c_double * 4) * 4), ("hole", C.c_double * 3),
                ("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)), ("metrics", C.POINTER(C.c_double))]


class ParamsC(C.Structure):
    _fields_ = [("d", C.c_int), ("C0", C.c_int), ("c_policy", C.c_int), ("gamma", C.c_double),
                ("alpha_f", C.c_double), ("p_f", C.c_int), ("cfl", C.c_double), ("n_f", C.c_int),
                ("n_v", C.c_int), ("win_r", C.c_int), ("loc", C.c_int), ("R", C.c_double * 4),
                ("depth_cap", C.c_int), ("fc_tables", C.POINTER(C.c_double)), ("fc_tables_len", C.c_int),
                ("sdnn_w", C.POINTER(C.c_float)), ("sdnn_len", C.c_int), ("freestream", C.c_double * 4),
                ("wall_form", C.c_int)]


# fc_comm_fn: (user, op, send_dev, send_counts, recv_dev, recv_counts, stream) -> int
COMM_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_longlong), C.c_void_p,
                      C.POINTER(C.c_longlong), C.c_void_p)
COMM_EXCHANGE, COMM_MIN = 0, 1


def library_path():
    return _LIBPATH


def load():
    """Load libfcsdnn.so (building it first if the sources are newer); raise if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        from . import build
        build.build()
    lib = C.CDLL(_LIBPATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    sig = {
        "fc_init_patches": (C.c_int, [C.POINTER(vp), C.POINTER(PatchDescC), ip, C.POINTER(ParamsC), vp]),
        "fc_state_size": (C.c_size_t, [vp]),
        "fc_active_points": (C.c_size_t, [vp]),
        "fc_patch_offset": (C.c_int, [vp, ip, C.POINTER(C.c_size_t)]),
        "fc_rhs": (C.c_int, [vp, vp, vp, vp, vp]),
        "fc_viscosity": (C.c_int, [vp, vp, vp, vp, vp]),
        "fc_filter": (C.c_int, [vp, vp, vp]),
        "fc_project": (C.c_int, [vp, vp, vp]),
        "fc_timestep": (C.c_int, [vp, vp, vp, vp, vp]),
        "fc_rk_step": (C.c_int, [vp, vp, vp, vp, ip, vp]),
        "fc_rk_step_host": (C.c_int, [vp, vp, vp, vp, ip, vp]),
        "fc_autotune": (C.c_int, [vp, ip, C.POINTER(C.c_double), vp]),
        "fc_adjoint_step": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, C.c_int, vp]),
        "fc_initial_sensitivity": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "fc_drag": (C.c_int, [vp, vp, vp, vp, vp]),
        "fc_sync_status": (C.c_int, [vp, vp, ip, vp]),
        "fc_launch_count": (C.c_uint64, [vp]),
        "fc_profile_enable": (C.c_int, [vp, ip]),
        "fc_profile_read": (C.c_int, [vp]),
        "fc_profile_get": (C.c_int, [vp, ip, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
        "fc_profile_reset": (C.c_int, [vp]),
        "fc_pass_stats": (C.c_int, [vp, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "fc_line_stats": (C.c_int, [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), ip]),
        "fc_probe_fp64": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), vp]),
        "fc_partition": (C.c_int, [C.POINTER(PatchDescC), ip, ip, C.POINTER(C.c_int)]),
        "fc_shard": (C.c_int, [vp, ip, ip, C.POINTER(C.c_int), COMM_FN, vp]),
        "fc_shard_counts": (C.c_int, [vp, ip, ip, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "fc_rhs_patch_noalloc": (C.c_int, [vp, vp, vp, ip, ip, C.POINTER(C.c_double), ip, ip,
                                           C.POINTER(C.c_double), ip, C.c_double, vp]),
        "fc_last_error": (C.c_char_p, [vp]),
        "fc_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


@functools.lru_cache(maxsize=None)
def fc_table_blob(d):
    """Pack fc_tables_d{d}.txt as the fc_params.fc_tables array: d, Cmin, Cmax, then Q, A_l, A_r per C."""
    path = os.path.join(_HERE, "data", f"fc_tables_d{d}.txt")
    with open(path) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    blocks, i = [], 0
    while lines[i] != "end":
        c = int(lines[i + 1].split()[1])
        i += 2
        rows = []
        for name, nr in (("Q", d), ("AL", c), ("AR", c)):
            assert lines[i] == name
            rows += [float(v) for r in range(nr) for v in lines[i + 1 + r].split()]
            i += 1 + nr
        blocks.append((c, rows))
    blocks.sort()
    cs = [c for c, _ in blocks]
    assert cs == list(range(cs[0], cs[-1] + 1))
    out = [float(d), float(cs[0]), float(cs[-1])]
    for _, rows in blocks:
        out += rows
    return np.array(out, dtype=np.float64)


@functools.lru_cache(maxsize=None)
def sdnn_blob():
    """fc_params.sdnn_w: W1, b1, W2, b2, W3, b3 of the stand-in classifier (FP32)."""
    path = os.path.join(_HERE, "data", "sdnn_standin.txt")
    with open(path) as f:
        lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    vals, i = [], 0
    while i < len(lines):
        r = int(lines[i][1])
        vals += [float(v) for k in range(r) for v in lines[i + 1 + k]]
        i += 1 + r
    return np.array(vals, dtype=np.float32)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def pack_descs(workload):
    """fc_patch_desc array of a workload, and the host arrays it points to (keep them alive)."""
    n = len(workload.patches)
    descs = (PatchDescC * n)()
    keep = []
    for k, p in enumerate(workload.patches):
        dsc = descs[k]
        dsc.kind, dsc.n1, dsc.n2 = p.kind, p.n1, p.n2
        for m in range(4):
            dsc.geom[m] = p.geom[m]
            dsc.side[m] = p.side[m]
            for q in range(4):
                dsc.bc[m][q] = p.bc[m][q]
        for m in range(3):
            dsc.hole[m] = p.hole[m]
        if p.kind == W.GRID:  # host arrays, kept alive until fc_init_patches returns
            ptrs = []
            for a, m in ((p.x, 1), (p.y, 1), (p.metrics, 4)):
                if a is None:  # null: metrics are then computed by the library; x, y are required
                    ptrs.append(None)
                    continue
                a = np.ascontiguousarray(a, dtype=np.float64)
                if a.size != m * p.n1 * p.n2:
                    raise ValueError(f"GRID patch {k}: array of {a.size} values, expected {m * p.n1 * p.n2}")
                keep.append(a)
                ptrs.append(a.ctypes.data_as(C.POINTER(C.c_double)))
            dsc.x, dsc.y, dsc.metrics = ptrs
    return descs, keep


def partition(workload, nranks):
    """fc_partition: owner rank of every patch (Morton order, balanced active points)."""
    lib = load()
    descs, keep = pack_descs(workload)
    n = len(workload.patches)
    owner = (C.c_int * n)()
    st = lib.fc_partition(descs, n, int(nranks), owner)
    if st != FC_OK:
        raise FcError(st, "fc_partition failed")
    return list(owner)


class _DevArray:
    """A device buffer owned by the library, seen by torch without a copy."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr or 0), False),
                                         "version": 3}


def _dev_tensor(ptr, n):
    import torch
    if n == 0:
        return torch.empty(0, dtype=torch.float64, device="cuda")
    return torch.as_tensor(_DevArray(ptr, n), device="cuda")


class Context:
    """One fc_ctx: geometry and device workspaces of a workload.

    States are device tensors of 4 * P doubles in the library's layout (component-major,
    patches concatenated in workload order, each row-major with q1 fastest); every call
    runs on the current torch stream."""

    def __init__(self, workload: W.Workload):
        lib = load()
        self.lib = lib
        self.w = workload
        prm = workload.params
        n = len(workload.patches)
        descs, keep = pack_descs(workload)
        self._tab = fc_table_blob(prm.d)
        self._sd = sdnn_blob()
        P = ParamsC()
        P.d, P.C0, P.c_policy, P.gamma, P.alpha_f, P.p_f = prm.d, prm.C0, prm.c_policy, prm.gamma, prm.alpha_f, prm.p_f
        P.cfl, P.n_f, P.n_v, P.win_r, P.loc, P.depth_cap = prm.cfl, prm.n_f, prm.n_v, prm.win_r, prm.loc, prm.depth_cap
        for m in range(4):
            P.R[m] = prm.R[m]
        P.fc_tables = self._tab.ctypes.data_as(C.POINTER(C.c_double))
        P.fc_tables_len = len(self._tab)
        P.sdnn_w = self._sd.ctypes.data_as(C.POINTER(C.c_float))
        P.sdnn_len = len(self._sd)
        for m in range(4):
            P.freestream[m] = workload.freestream[m]
        P.wall_form = getattr(prm, "wall_form", 0)
        ctx = C.c_void_p()
        st = lib.fc_init_patches(C.byref(ctx), descs, n, C.byref(P), None)
        if st != FC_OK:
            raise FcError(st, "fc_init_patches failed (see stderr)")
        self.ctx = ctx
        self.P = lib.fc_state_size(ctx)
        self.active = lib.fc_active_points(ctx)

    def __del__(self):
        if getattr(self, "ctx", None):
            self.lib.fc_destroy(self.ctx)
            self.ctx = None

    def _check(self, st):
        if st != FC_OK:
            raise FcError(st, self.lib.fc_last_error(self.ctx).decode())

    def offsets(self):
        out = []
        for k in range(len(self.w.patches)):
            o = C.c_size_t()
            self._check(self.lib.fc_patch_offset(self.ctx, k, C.byref(o)))
            out.append(o.value)
        return out

    def rhs(self, e, out, mu=None):
        self._check(self.lib.fc_rhs(self.ctx, _ptr(e), _ptr(out), _ptr(mu), _stream()))

    def viscosity(self, e, mu, tau=None):
        self._check(self.lib.fc_viscosity(self.ctx, _ptr(e), _ptr(mu), _ptr(tau), _stream()))

    def filter(self, e):
        self._check(self.lib.fc_filter(self.ctx, _ptr(e), _stream()))

    def project(self, e):
        self._check(self.lib.fc_project(self.ctx, _ptr(e), _stream()))

    def timestep(self, e, mu, dt):
        self._check(self.lib.fc_timestep(self.ctx, _ptr(e), _ptr(mu), _ptr(dt), _stream()))

    def rk_step(self, e, dt, mu, flags=0):
        self._check(self.lib.fc_rk_step(self.ctx, _ptr(e), _ptr(dt), _ptr(mu), int(flags), _stream()))

    def rk_step_host(self, e_host, dt, mu, flags=0):
        """fc_rk_step_host: one step of a state in host memory (a contiguous CPU float64 tensor
        of 4 P values, best page-locked); returns when e_host holds the new state."""
        import torch
        if not (isinstance(e_host, torch.Tensor) and not e_host.is_cuda and e_host.dtype == torch.float64
                and e_host.is_contiguous() and e_host.numel() == 4 * self.P):
            raise FcError(FC_ERR_INVALID, f"e_host must be a contiguous CPU float64 tensor of {4 * self.P} values")
        self._check(self.lib.fc_rk_step_host(self.ctx, C.c_void_p(e_host.data_ptr()), _ptr(dt), _ptr(mu),
                                             int(flags), _stream()))

    def autotune(self, flags=TUNE_PLANS | TUNE_WARPS):
        """Measured choice of FFT stage orders and warps per CTA (fc_autotune); returns its report."""
        rep = (C.c_double * 6)()
        self._check(self.lib.fc_autotune(self.ctx, int(flags), rep, _stream()))
        keys = ("lengths", "lengths_changed", "classes", "classes_changed", "ms_before", "ms_after")
        return {k: (int(v) if k[0] in "lc" else float(v)) for k, v in zip(keys, rep)}

    def adjoint_step(self, e_n, mu, dt, lam_np1, lam_n, gbc=None, flags=0, dparam=None):
        """fc_adjoint_step; dparam (2 device doubles) accumulates dJ/d(Mach, angle) through the
        free-stream Dirichlet states."""
        self._check(self.lib.fc_adjoint_step(self.ctx, _ptr(e_n), _ptr(mu), _ptr(dt), _ptr(lam_np1), _ptr(lam_n),
                                             _ptr(gbc), _ptr(dparam), int(flags), _stream()))

    def initial_sensitivity(self, e0, lam0, drho=None, dparam=None):
        """fc_initial_sensitivity: dJ/drho_0 into drho (P doubles) and, for a uniform free-stream
        e0, its dJ/d(Mach, angle) part accumulated into dparam (2 doubles)."""
        self._check(self.lib.fc_initial_sensitivity(self.ctx, _ptr(e0), _ptr(lam0), _ptr(drho), _ptr(dparam),
                                                    _stream()))

    def shard(self, nranks, rank, owner, comm):
        """fc_shard: this context becomes rank `rank` of nranks with the patch owners `owner`;
        comm has exchange(send, send_counts, recv, recv_counts) (an all-to-all of device
        tensors with those splits) and allmin(send, recv), both ordered on the current stream."""
        import torch
        nr = int(nranks)

        def cb(user, op, send, scounts, recv, rcounts, stream):
            try:
                s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(s):
                    if op == COMM_MIN:
                        comm.allmin(_dev_tensor(send, 1), _dev_tensor(recv, 1))
                    else:
                        sc = [int(scounts[q]) for q in range(nr)]
                        rc = [int(rcounts[q]) for q in range(nr)]
                        comm.exchange(_dev_tensor(send, sum(sc)), sc, _dev_tensor(recv, sum(rc)), rc)
                return 0
            except Exception:  # reported to the library as a failed exchange
                import traceback
                traceback.print_exc()
                return 1

        self._comm_cb = COMM_FN(cb)  # kept alive with the context
        self._comm = comm
        own = (C.c_int * len(self.w.patches))(*owner)
        self._check(self.lib.fc_shard(self.ctx, nr, int(rank), own, self._comm_cb, None))
        self.nranks, self.rank, self.owner = nr, int(rank), list(owner)

    def shard_counts(self, which, peer):
        """(doubles sent to, received from) peer per exchange: which 0 fringe, 1 viscosity."""
        a, b = C.c_longlong(), C.c_longlong()
        self._check(self.lib.fc_shard_counts(self.ctx, int(which), int(peer), C.byref(a), C.byref(b)))
        return a.value, b.value

    def drag(self, e, J, dJde=None):
        self._check(self.lib.fc_drag(self.ctx, _ptr(e), _ptr(J), _ptr(dJde), _stream()))

    def sync_status(self, e=None, check_state=True):
        return self.lib.fc_sync_status(self.ctx, _ptr(e), 1 if (check_state and e is not None) else 0, _stream())

    def launch_count(self):
        return int(self.lib.fc_launch_count(self.ctx))

    def profile(self, enable=True):
        self._check(self.lib.fc_profile_enable(self.ctx, 1 if enable else 0))

    def profile_read(self):
        """{group name: (total ms, launches)} of the instrumented calls since the last reset."""
        n = self.lib.fc_profile_read(self.ctx)
        if n < 0:
            raise FcError(2, "fc_profile_read failed")
        out = {}
        for k in range(n):
            nm, ms, cnt = C.c_char_p(), C.c_double(), C.c_int()
            self._check(self.lib.fc_profile_get(self.ctx, k, C.byref(nm), C.byref(ms), C.byref(cnt)))
            out[nm.value.decode()] = (ms.value, cnt.value)
        return out

    def pass_stats(self, name):
        """(algorithmic FP64 flops, compulsory bytes, lines, points) of one launch of a line pass."""
        f, b, nl, npt = C.c_double(), C.c_double(), C.c_longlong(), C.c_longlong()
        self._check(self.lib.fc_pass_stats(self.ctx, name.encode(), C.byref(f), C.byref(b), C.byref(nl),
                                           C.byref(npt)))
        return f.value, b.value, nl.value, npt.value

    def line_stats(self, reset=True):
        """(skipped q1 lines, skipped q2 lines, skipped q1 flops, skipped q2 flops) since the last reset."""
        a, b, f, g = C.c_longlong(), C.c_longlong(), C.c_double(), C.c_double()
        self._check(self.lib.fc_line_stats(self.ctx, C.byref(a), C.byref(b), C.byref(f), C.byref(g), 1 if reset else 0))
        return a.value, b.value, f.value, g.value

    def profile_reset(self):
        self._check(self.lib.fc_profile_reset(self.ctx))


def probe_fp64():
    """(DFMA, DMMA) FP64 rates of the current device in GFLOP/s (fc_probe_fp64)."""
    lib = load()
    a, b = C.c_double(), C.c_double()
    st = lib.fc_probe_fp64(C.byref(a), C.byref(b), _stream())
    if st != FC_OK:
        raise FcError(st, "fc_probe_fp64 failed")
    return a.value, b.value


def _check_field(t, name, numel):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and t.numel() == numel):
        raise FcError(FC_ERR_INVALID, f"{name} must be a contiguous CUDA float64 tensor of {numel} elements")


def rhs_patch_noalloc(e, mu, out, n1, n2, box, d, ncont, gamma=W.GAMMA):
    """fc_rhs_patch_noalloc: RHS of one stand-alone affine patch, no device allocation."""
    lib = load()
    n1, n2, d, ncont = int(n1), int(n2), int(d), int(ncont)
    tab = fc_table_blob(d)
    cmin, cmax = int(tab[1]), int(tab[2])
    if not cmin <= ncont <= cmax:
        raise FcError(FC_ERR_INVALID, f"C = {ncont} is outside the tabulated range [{cmin}, {cmax}] for d = {d}")
    if n1 <= 0 or n2 <= 0:
        raise FcError(FC_ERR_INVALID, f"bad patch size {n1} x {n2}")
    _check_field(e, "e", 4 * n1 * n2)
    _check_field(out, "out", 4 * n1 * n2)
    _check_field(mu, "mu", n1 * n2)
    off = 3 + sum(d * d + 2 * c * d for c in range(cmin, ncont))
    block = np.ascontiguousarray(tab[off:off + d * d + 2 * ncont * d])
    bx = np.ascontiguousarray(np.asarray(box, dtype=np.float64))
    if bx.shape != (4,):
        raise FcError(FC_ERR_INVALID, "box must hold (x0, x1, y0, y1)")
    st = lib.fc_rhs_patch_noalloc(_ptr(e), _ptr(mu), _ptr(out), n1, n2,
                                  bx.ctypes.data_as(C.POINTER(C.c_double)), d, ncont,
                                  block.ctypes.data_as(C.POINTER(C.c_double)), int(block.size), float(gamma),
                                  _stream())
    if st != FC_OK:
        raise FcError(st, "fc_rhs_patch_noalloc failed (see stderr)")
