"""ctypes binding of the solver's C ABI (include/ibm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. PyTorch provides the device workspace (so the memory belongs to
torch's caching allocator) and the CUDA stream. The library must have been
built (``paper_2103_08246_gb300.build.build()``); loading fails loudly
otherwise, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .inputs import Workload

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibm_gb300.so")

IBM_OK, IBM_EINVAL, IBM_ENOMEM, IBM_ECUDA, IBM_EDIVERGED, IBM_ETIMEOUT, IBM_EIO = 0, -1, -2, -3, -4, -5, -6
IBM_FP64, IBM_FP32, IBM_MIXED = 0, 1, 2
IBM_FIELD_U, IBM_FIELD_V, IBM_FIELD_W, IBM_FIELD_P = 0, 1, 2, 3

# every symbol include/ibm.h declares
SYMBOLS = ("ibm_workspace_bytes", "ibm_create", "ibm_step", "ibm_sync", "ibm_flag_state",
           "ibm_stats", "ibm_get_field", "ibm_set_field", "ibm_marker_count", "ibm_get_markers",
           "ibm_save", "ibm_load", "ibm_set_inflow", "ibm_inflow_planes", "ibm_get_plane",
           "ibm_plane_device", "ibm_probes_set", "ibm_probe_sample",
           "ibm_time_stage", "ibm_stats_static", "ibm_ensemble_create", "ibm_ensemble_create_batched",
           "ibm_ensemble_step", "ibm_ensemble_destroy",
           "ibm_gen_create", "ibm_gen_param_count", "ibm_gen_set_params", "ibm_gen_get_params",
           "ibm_gen_get_grads", "ibm_gen_set_norm", "ibm_gen_forward", "ibm_gen_grad", "ibm_gen_adam_step",
           "ibm_gen_train_step", "ibm_gen_train_step_pushforward", "ibm_gen_eval", "ibm_gen_set_noise",
           "ibm_gen_set_relax",
           "ibm_gen_set_spectrum", "ibm_gen_set_lr", "ibm_gen_time", "ibm_gen_rollout_init",
           "ibm_gen_rollout", "ibm_gen_emit", "ibm_gen_history", "ibm_gen_save", "ibm_gen_load", "ibm_gen_sync",
           "ibm_gen_destroy", "ibm_check_bounded_wait", "ibm_destroy", "ibm_strerror",
           "ibm_slab_ghosts", "ibm_slab_split", "ibm_slab_plan", "ibm_create_slab", "ibm_slab_workspace_bytes",
           "ibm_slab_phase")
_VOID = ("ibm_destroy", "ibm_ensemble_destroy", "ibm_gen_destroy")

IBM_SLAB_INIT, IBM_SLAB_FORCE, IBM_SLAB_SOLVE, IBM_SLAB_REDUCE, IBM_SLAB_PROJECT, IBM_SLAB_GHOSTS = range(6)
IBM_XCHG_NONE, IBM_XCHG_SUM, IBM_XCHG_GATHER, IBM_XCHG_HALO = range(4)
IBM_SLAB_MAX_RANKS = 8

STAGES = {"step": -1, "rhs": 0, "outflow": 1, "af_x": 2, "af_y": 3, "af_z": 4, "ib": 5, "flag": 6,
          "mass_div": 7, "dht_y": 8, "dht_z": 9, "poisson_x": 10, "project": 11, "poisson": 12,
          "af_yz": 13, "dht2d": 14, "tc_pass": 15, "residual": 16, "tc_pass1": 17, "tc_bf16": 18,
          "poisson_x16": 19}


class ibm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class ibm_domain(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class ibm_bodies(ctypes.Structure):
    _fields_ = [("bars_on", ctypes.c_int), ("bar_x", ctypes.c_double),
                ("bar_mesh", ctypes.c_double), ("bar_width", ctypes.c_double),
                ("flag_on", ctypes.c_int), ("flag_x_le", ctypes.c_double),
                ("flag_len", ctypes.c_double), ("flag_span", ctypes.c_double),
                ("flag_ns", ctypes.c_int), ("flag_nt", ctypes.c_int),
                ("mass_ratio", ctypes.c_double), ("bending", ctypes.c_double),
                ("pitch0", ctypes.c_double), ("stretch", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)


class ibm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cfl", ctypes.c_double),
                ("cfl_limit", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("init_u", _dp), ("init_v", _dp), ("init_w", _dp),
                ("rhs_planes", ctypes.c_int), ("afx_planes", ctypes.c_int),
                ("rhs_stages", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("inflow", ctypes.c_int), ("bar_forcing", ctypes.c_int),
                ("mixed_tc_predictor", ctypes.c_int)]


class ibm_slab(ctypes.Structure):
    _fields_ = [("nranks", ctypes.c_int), ("rank", ctypes.c_int), ("x_begin", ctypes.c_int),
                ("x_end", ctypes.c_int), ("ghosts", ctypes.c_int)]


class ibm_gen_config(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nz", ctypes.c_int), ("width", ctypes.c_int),
                ("blocks", ctypes.c_int), ("in_channels", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("stream", ctypes.c_void_p), ("stride", ctypes.c_int)]


class ibm_stats_t(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("cfl", ctypes.c_double), ("max_div", ctypes.c_double),
                ("q_in", ctypes.c_double), ("q_out", ctypes.c_double), ("ke", ctypes.c_double),
                ("ib_slip", ctypes.c_double), ("te_mid", ctypes.c_double * 3),
                ("force", ctypes.c_double * 3), ("max_strain", ctypes.c_double),
                ("n_sub", ctypes.c_int), ("n_markers", ctypes.c_int),
                ("kernels_per_step", ctypes.c_int)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"solver library not built: {path} is missing "
                           "(run paper_2103_08246_gb300.build.build())")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    sz = ctypes.c_size_t
    lib.ibm_workspace_bytes.argtypes = [ctypes.POINTER(ibm_grid), ctypes.POINTER(ibm_domain),
                                        ctypes.POINTER(ibm_bodies), ctypes.POINTER(ibm_options),
                                        ctypes.POINTER(sz)]
    lib.ibm_create.argtypes = [ctypes.POINTER(ibm_grid), ctypes.POINTER(ibm_domain), ctypes.c_double,
                               ctypes.POINTER(ibm_bodies), ctypes.POINTER(ibm_options), vp, sz,
                               ctypes.POINTER(vp)]
    lib.ibm_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    lib.ibm_sync.argtypes = [vp]
    lib.ibm_check_bounded_wait.argtypes = [ctypes.c_uint]
    lib.ibm_flag_state.argtypes = [vp, _dp, _dp, _dp, sz]
    lib.ibm_stats.argtypes = [vp, ctypes.POINTER(ibm_stats_t)]
    lib.ibm_stats_static.argtypes = [vp, ctypes.POINTER(ibm_stats_t)]
    lib.ibm_get_field.argtypes = [vp, ctypes.c_int, _dp, sz]
    lib.ibm_set_field.argtypes = [vp, ctypes.c_int, _dp, sz]
    lib.ibm_marker_count.argtypes = [vp, ctypes.POINTER(sz)]
    lib.ibm_get_markers.argtypes = [vp, _dp, sz]
    lib.ibm_set_inflow.argtypes = [vp, _dp, _dp, _dp]
    lib.ibm_get_plane.argtypes = [vp, ctypes.c_int, _dp, _dp, _dp]
    lib.ibm_plane_device.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp)]
    lib.ibm_inflow_planes.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.ibm_probes_set.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.ibm_probe_sample.argtypes = [vp, vp]
    lib.ibm_save.argtypes = [vp, ctypes.c_char_p]
    lib.ibm_load.argtypes = [vp, ctypes.c_char_p]
    lib.ibm_time_stage.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.ibm_ensemble_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.ibm_ensemble_create_batched.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.ibm_ensemble_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    lib.ibm_ensemble_destroy.argtypes = [vp]
    lib.ibm_destroy.argtypes = [vp]
    lib.ibm_strerror.argtypes = [ctypes.c_int]
    lib.ibm_strerror.restype = ctypes.c_char_p
    ip = ctypes.POINTER(ctypes.c_int)
    slp = ctypes.POINTER(ibm_slab)
    lib.ibm_slab_ghosts.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ip]
    lib.ibm_slab_split.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, slp]
    lib.ibm_slab_plan.argtypes = [ctypes.POINTER(ibm_grid), ctypes.c_int, slp, ctypes.c_int, ip,
                                  ctypes.POINTER(sz), ctypes.POINTER(sz)]
    lib.ibm_create_slab.argtypes = [ctypes.POINTER(ibm_grid), ctypes.POINTER(ibm_domain), ctypes.c_double,
                                    ctypes.POINTER(ibm_bodies), ctypes.POINTER(ibm_options), slp, vp, sz,
                                    ctypes.POINTER(vp)]
    lib.ibm_slab_workspace_bytes.argtypes = [ctypes.POINTER(ibm_grid), ctypes.POINTER(ibm_domain),
                                             ctypes.POINTER(ibm_bodies), ctypes.POINTER(ibm_options), slp,
                                             ctypes.POINTER(sz)]
    lib.ibm_slab_phase.argtypes = [vp, ctypes.c_int, ctypes.c_double, vp, vp]
    lib.ibm_gen_create.argtypes = [ctypes.POINTER(ibm_gen_config), ctypes.POINTER(vp)]
    lib.ibm_gen_param_count.argtypes = [vp]
    lib.ibm_gen_set_params.argtypes = [vp, _dp, sz]
    lib.ibm_gen_get_params.argtypes = [vp, _dp, sz]
    lib.ibm_gen_get_grads.argtypes = [vp, _dp, sz]
    lib.ibm_gen_set_norm.argtypes = [vp, _dp, _dp, _dp]
    lib.ibm_gen_forward.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    lib.ibm_gen_grad.argtypes = [vp, vp, vp, vp, ctypes.c_int, _dp]
    lib.ibm_gen_adam_step.argtypes = [vp]
    lib.ibm_gen_train_step.argtypes = [vp, vp, ctypes.c_int, ip, ctypes.c_int, _dp]
    lib.ibm_gen_train_step_pushforward.argtypes = [vp, vp, ctypes.c_int, ip, ctypes.c_int, _dp]
    lib.ibm_gen_eval.argtypes = [vp, vp, ctypes.c_int, ip, ctypes.c_int, _dp]
    lib.ibm_gen_set_lr.argtypes = [vp, ctypes.c_double]
    lib.ibm_gen_set_noise.argtypes = [vp, ctypes.c_double, ctypes.c_ulonglong]
    lib.ibm_gen_set_relax.argtypes = [vp, _dp, ctypes.c_double]
    lib.ibm_gen_set_spectrum.argtypes = [vp, _dp, ctypes.c_double]
    lib.ibm_gen_time.argtypes = [vp, ctypes.c_int, ctypes.c_int, _dp]
    lib.ibm_gen_rollout_init.argtypes = [vp, vp, vp]
    lib.ibm_gen_rollout.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    lib.ibm_gen_history.argtypes = [vp, vp, vp]
    lib.ibm_gen_emit.argtypes = [vp, ctypes.c_double, vp, vp, vp, ctypes.c_int]
    lib.ibm_gen_sync.argtypes = [vp]
    lib.ibm_gen_save.argtypes = [vp, ctypes.c_char_p]
    lib.ibm_gen_load.argtypes = [vp, ctypes.c_char_p]
    lib.ibm_gen_destroy.argtypes = [vp]
    for name in SYMBOLS:
        if name in _VOID:
            getattr(lib, name).restype = None
        elif name != "ibm_strerror":
            getattr(lib, name).restype = ctypes.c_int
    lib.ibm_gen_param_count.restype = sz
    _lib = lib
    return lib


class IBMError(RuntimeError):
    def __init__(self, code, where):
        msg = load().ibm_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def _check(code, where):
    if code != IBM_OK:
        raise IBMError(code, where)


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def structs_from_workload(wl: Workload):
    grid = ibm_grid(wl.nx, wl.ny, wl.nz)
    dom = ibm_domain(wl.lx, wl.ly, wl.lz)
    bodies = ibm_bodies(int(wl.bars_on), wl.bar_x, wl.bar_mesh, wl.bar_width, int(wl.flag_on),
                        wl.flag_x_le, wl.flag_len, wl.flag_span, wl.flag_ns, wl.flag_nt,
                        wl.mass_ratio, wl.bending, wl.pitch0, wl.stretch)
    return grid, dom, bodies


# ----------------------------------------------------------------- C-ABI names
def ibm_workspace_bytes(grid, dom, bodies, opts) -> int:
    n = ctypes.c_size_t(0)
    _check(load().ibm_workspace_bytes(ctypes.byref(grid), ctypes.byref(dom), ctypes.byref(bodies),
                                      ctypes.byref(opts) if opts is not None else None,
                                      ctypes.byref(n)), "ibm_workspace_bytes")
    return n.value


def ibm_create(grid, dom, re, bodies, opts, workspace_ptr=None, workspace_bytes=0):
    h = ctypes.c_void_p()
    _check(load().ibm_create(ctypes.byref(grid), ctypes.byref(dom), float(re), ctypes.byref(bodies),
                             ctypes.byref(opts) if opts is not None else None,
                             workspace_ptr, workspace_bytes, ctypes.byref(h)), "ibm_create")
    return h


def ibm_slab_ghosts(re, h, dt) -> int:
    g = ctypes.c_int(0)
    _check(load().ibm_slab_ghosts(float(re), float(h), float(dt), ctypes.byref(g)), "ibm_slab_ghosts")
    return g.value


def ibm_slab_split(nx, nranks, rank, ghosts) -> ibm_slab:
    out = ibm_slab()
    _check(load().ibm_slab_split(int(nx), int(nranks), int(rank), int(ghosts), ctypes.byref(out)),
           "ibm_slab_split")
    return out


def ibm_slab_plan(grid, n_flag_vertices, slab, phase):
    """(exchange kind, send count, recv count) of a phase."""
    k = ctypes.c_int(0)
    ns, nr = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(load().ibm_slab_plan(ctypes.byref(grid), int(n_flag_vertices), ctypes.byref(slab), int(phase),
                                ctypes.byref(k), ctypes.byref(ns), ctypes.byref(nr)), "ibm_slab_plan")
    return k.value, ns.value, nr.value


def ibm_slab_workspace_bytes(grid, dom, bodies, opts, slab) -> int:
    n = ctypes.c_size_t(0)
    _check(load().ibm_slab_workspace_bytes(ctypes.byref(grid), ctypes.byref(dom), ctypes.byref(bodies),
                                           ctypes.byref(opts) if opts is not None else None,
                                           ctypes.byref(slab), ctypes.byref(n)), "ibm_slab_workspace_bytes")
    return n.value


def ibm_create_slab(grid, dom, re, bodies, opts, slab, workspace_ptr=None, workspace_bytes=0):
    h = ctypes.c_void_p()
    _check(load().ibm_create_slab(ctypes.byref(grid), ctypes.byref(dom), float(re), ctypes.byref(bodies),
                                  ctypes.byref(opts) if opts is not None else None, ctypes.byref(slab),
                                  workspace_ptr, workspace_bytes, ctypes.byref(h)), "ibm_create_slab")
    return h


def ibm_slab_phase(state, phase, dt, recv_ptr, send_ptr):
    return load().ibm_slab_phase(state, int(phase), float(dt), recv_ptr, send_ptr)


def ibm_step(state, dt, nsteps):
    return load().ibm_step(state, float(dt), int(nsteps))


def ibm_sync(state):
    _check(load().ibm_sync(state), "ibm_sync")


def ibm_check_bounded_wait(spins):
    """Status of the bounded-wait self-test (IBM_ETIMEOUT expected)."""
    return load().ibm_check_bounded_wait(int(spins))


def ibm_flag_state(state, X, V=None, F=None):
    _check(load().ibm_flag_state(state, _ptr(X), _ptr(V), _ptr(F), X.size // 3), "ibm_flag_state")


def ibm_stats(state) -> dict:
    st = ibm_stats_t()
    _check(load().ibm_stats(state, ctypes.byref(st)), "ibm_stats")
    return st.as_dict()


def ibm_stats_static(state) -> dict:
    """Diagnostics through the entry point that allocates nothing."""
    st = ibm_stats_t()
    _check(load().ibm_stats_static(state, ctypes.byref(st)), "ibm_stats_static")
    return st.as_dict()


def ibm_get_field(state, which, out):
    _check(load().ibm_get_field(state, which, _ptr(out), out.size), "ibm_get_field")


def ibm_set_field(state, which, arr):
    a = np.ascontiguousarray(arr, dtype=np.float64)
    _check(load().ibm_set_field(state, which, _ptr(a), a.size), "ibm_set_field")


def ibm_marker_count(state) -> int:
    n = ctypes.c_size_t(0)
    _check(load().ibm_marker_count(state, ctypes.byref(n)), "ibm_marker_count")
    return n.value


def ibm_get_markers(state, out):
    _check(load().ibm_get_markers(state, _ptr(out), out.size // 3), "ibm_get_markers")


def ibm_set_inflow(state, u, v, w):
    a = [np.ascontiguousarray(q, dtype=np.float64) for q in (u, v, w)]
    _check(load().ibm_set_inflow(state, *[_ptr(q) for q in a]), "ibm_set_inflow")


def ibm_get_plane(state, i, u, v, w):
    _check(load().ibm_get_plane(state, int(i), _ptr(u), _ptr(v), _ptr(w)), "ibm_get_plane")


def ibm_plane_device(state, i):
    """Device addresses of x-plane i of u, v, w (valid until the next step)."""
    ptrs = [ctypes.c_void_p() for _ in range(3)]
    _check(load().ibm_plane_device(state, int(i), *[ctypes.byref(q) for q in ptrs]),
           "ibm_plane_device")
    return tuple(q.value for q in ptrs)


def ibm_inflow_planes(state):
    """Device addresses of the pending inflow planes (u, v, w)."""
    ptrs = [ctypes.c_void_p() for _ in range(3)]
    _check(load().ibm_inflow_planes(state, *[ctypes.byref(q) for q in ptrs]), "ibm_inflow_planes")
    return tuple(q.value for q in ptrs)


def ibm_probes_set(state, ijk):
    a = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    _check(load().ibm_probes_set(state, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), a.shape[0]),
           "ibm_probes_set")


def ibm_probe_sample(state, dst):
    _check(load().ibm_probe_sample(state, dst), "ibm_probe_sample")


def ibm_save(state, path):
    _check(load().ibm_save(state, os.fsencode(path)), "ibm_save")


def ibm_load(state, path):
    _check(load().ibm_load(state, os.fsencode(path)), "ibm_load")


def ibm_time_stage(state, stage, nrep) -> float:
    ms = ctypes.c_double(0.0)
    _check(load().ibm_time_stage(state, int(stage), int(nrep), ctypes.byref(ms)), "ibm_time_stage")
    return ms.value


def ibm_ensemble_create(states, stream=None, batched=False):
    arr = (ctypes.c_void_p * len(states))(*[st.value if isinstance(st, ctypes.c_void_p) else st
                                             for st in states])
    h = ctypes.c_void_p()
    name = "ibm_ensemble_create_batched" if batched else "ibm_ensemble_create"
    _check(getattr(load(), name)(arr, len(states), stream, ctypes.byref(h)), name)
    return h


def ibm_ensemble_step(ens, dt, nsteps):
    return load().ibm_ensemble_step(ens, float(dt), int(nsteps))


def ibm_ensemble_destroy(ens):
    load().ibm_ensemble_destroy(ens)


def ibm_destroy(state):
    load().ibm_destroy(state)


def ibm_gen_create(cfg):
    h = ctypes.c_void_p()
    _check(load().ibm_gen_create(ctypes.byref(cfg), ctypes.byref(h)), "ibm_gen_create")
    return h


def ibm_gen_param_count(gen) -> int:
    return int(load().ibm_gen_param_count(gen))


def ibm_gen_set_params(gen, w):
    a = np.ascontiguousarray(w, dtype=np.float64)
    _check(load().ibm_gen_set_params(gen, _ptr(a), a.size), "ibm_gen_set_params")


def ibm_gen_get_params(gen, out):
    _check(load().ibm_gen_get_params(gen, _ptr(out), out.size), "ibm_gen_get_params")


def ibm_gen_get_grads(gen, out):
    _check(load().ibm_gen_get_grads(gen, _ptr(out), out.size), "ibm_gen_get_grads")


def ibm_gen_set_norm(gen, mean, std, rms):
    a = [np.ascontiguousarray(q, dtype=np.float64) for q in (mean, std, rms)]
    _check(load().ibm_gen_set_norm(gen, *[_ptr(q) for q in a]), "ibm_gen_set_norm")


def ibm_gen_forward(gen, q_t, q_prev, delta, batch):
    _check(load().ibm_gen_forward(gen, q_t, q_prev, delta, int(batch)), "ibm_gen_forward")


def ibm_gen_grad(gen, q_t, q_prev, target, batch) -> float:
    loss = ctypes.c_double(0.0)
    _check(load().ibm_gen_grad(gen, q_t, q_prev, target, int(batch), ctypes.byref(loss)), "ibm_gen_grad")
    return loss.value


def ibm_gen_adam_step(gen):
    _check(load().ibm_gen_adam_step(gen), "ibm_gen_adam_step")


def ibm_gen_train_step(gen, planes, n_planes, t_idx, with_loss=True):
    idx = np.ascontiguousarray(t_idx, dtype=np.int32)
    loss = ctypes.c_double(0.0)
    _check(load().ibm_gen_train_step(gen, planes, int(n_planes),
                                     idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), idx.size,
                                     ctypes.byref(loss) if with_loss else None), "ibm_gen_train_step")
    return loss.value if with_loss else None


def ibm_gen_train_step_pushforward(gen, planes, n_planes, t_idx, with_loss=True):
    idx = np.ascontiguousarray(t_idx, dtype=np.int32)
    loss = ctypes.c_double(0.0)
    _check(load().ibm_gen_train_step_pushforward(gen, planes, int(n_planes),
                                                 idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), idx.size,
                                                 ctypes.byref(loss) if with_loss else None),
           "ibm_gen_train_step_pushforward")
    return loss.value if with_loss else None


def ibm_gen_eval(gen, planes, n_planes, t_idx) -> float:
    idx = np.ascontiguousarray(t_idx, dtype=np.int32)
    loss = ctypes.c_double(0.0)
    _check(load().ibm_gen_eval(gen, planes, int(n_planes), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               idx.size, ctypes.byref(loss)), "ibm_gen_eval")
    return loss.value


def ibm_gen_set_noise(gen, std, seed=0):
    _check(load().ibm_gen_set_noise(gen, float(std), int(seed)), "ibm_gen_set_noise")


def ibm_gen_set_relax(gen, plane, lam):
    a = None if plane is None else np.ascontiguousarray(plane, dtype=np.float64)
    _check(load().ibm_gen_set_relax(gen, _ptr(a), float(lam)), "ibm_gen_set_relax")


def ibm_gen_set_spectrum(gen, power, lam):
    a = None if power is None else np.ascontiguousarray(power, dtype=np.float64)
    _check(load().ibm_gen_set_spectrum(gen, _ptr(a), float(lam)), "ibm_gen_set_spectrum")


def ibm_gen_set_lr(gen, lr):
    _check(load().ibm_gen_set_lr(gen, float(lr)), "ibm_gen_set_lr")


GEN_TIMINGS = {"train_step": 0, "forward": 1, "conv_fwd": 2, "conv_dgrad": 3, "conv_wgrad": 4}


def ibm_gen_time(gen, what, nrep) -> float:
    ms = ctypes.c_double(0.0)
    _check(load().ibm_gen_time(gen, int(what), int(nrep), ctypes.byref(ms)), "ibm_gen_time")
    return ms.value


def ibm_gen_rollout_init(gen, plane_prev, plane_cur):
    _check(load().ibm_gen_rollout_init(gen, plane_prev, plane_cur), "ibm_gen_rollout_init")


def ibm_gen_rollout(gen, u, v, w, precision):
    _check(load().ibm_gen_rollout(gen, u, v, w, int(precision)), "ibm_gen_rollout")


def ibm_gen_emit(gen, w, u, v, wv, precision):
    _check(load().ibm_gen_emit(gen, float(w), u, v, wv, int(precision)), "ibm_gen_emit")


def ibm_gen_history(gen, q_t, q_prev):
    _check(load().ibm_gen_history(gen, q_t, q_prev), "ibm_gen_history")


def ibm_gen_save(gen, path):
    _check(load().ibm_gen_save(gen, os.fsencode(path)), "ibm_gen_save")


def ibm_gen_load(gen, path):
    _check(load().ibm_gen_load(gen, os.fsencode(path)), "ibm_gen_load")


def ibm_gen_sync(gen):
    _check(load().ibm_gen_sync(gen), "ibm_gen_sync")


def ibm_gen_destroy(gen):
    load().ibm_gen_destroy(gen)


# ----------------------------------------------------------------- convenience
class Solver:
    """One solver state on the current CUDA device.

    The device workspace is a torch uint8 tensor (torch's caching allocator);
    the stream is torch's current stream unless one is given.
    """

    def __init__(self, wl: Workload, precision: int = IBM_FP64, noise=None, stream=None,
                 cfl: float | None = None, cfl_limit: float = 2.0, tiles=None,
                 deterministic: bool = False, inflow: bool = False, tc_predictor: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the solver needs a CUDA device")
        load()
        self.wl = wl
        self.precision = precision
        self.grid, self.dom, self.bodies = structs_from_workload(wl)
        # a dedicated stream: CUDA graphs cannot be captured on the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._noise = [np.ascontiguousarray(a, dtype=np.float64) for a in noise] if noise else None
        tiles = tiles or {}
        opts = ibm_options(precision, wl.cfl if cfl is None else cfl, cfl_limit,
                           ctypes.c_void_p(self.stream.cuda_stream),
                           *([_ptr(a) for a in self._noise] if self._noise else [None] * 3),
                           int(tiles.get("rhs_planes", 0)), int(tiles.get("afx_planes", 0)),
                           int(tiles.get("rhs_stages", 0)), 1 if deterministic else 0,
                           1 if inflow else 0, 1 if wl.bar_forcing == "eulerian" else 0,
                           1 if tc_predictor else 0)
        self.ws_bytes = ibm_workspace_bytes(self.grid, self.dom, self.bodies, opts)
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.state = ibm_create(self.grid, self.dom, wl.re, self.bodies, opts,
                                ctypes.c_void_p(aligned), self.ws_bytes)
        self.nf = wl.flag_ns * wl.flag_nt if wl.flag_on else 0

    def step(self, nsteps=1, dt=None):
        dt = self.wl.dt if dt is None else dt
        rc = ibm_step(self.state, dt if dt is not None else -1.0, nsteps)
        _check(rc, "ibm_step")

    def field(self, which):
        wl = self.wl
        planes = wl.nx if which == IBM_FIELD_P else wl.nx + 1
        out = np.empty((planes, wl.ny, wl.nz))
        ibm_get_field(self.state, which, out)
        return out

    def fields(self):
        return tuple(self.field(q) for q in (IBM_FIELD_U, IBM_FIELD_V, IBM_FIELD_W, IBM_FIELD_P))

    def flag(self):
        X = np.empty((self.nf, 3))
        V = np.empty((self.nf, 3))
        F = np.empty((self.nf, 3))
        ibm_flag_state(self.state, X, V, F)
        return X, V, F

    def markers(self):
        n = ibm_marker_count(self.state)
        X = np.empty((n, 3))
        ibm_get_markers(self.state, X)
        return X

    def stats(self):
        return ibm_stats(self.state)

    def set_inflow(self, u, v, w):
        ibm_set_inflow(self.state, u, v, w)

    def plane(self, i):
        wl = self.wl
        out = [np.empty((wl.ny, wl.nz)) for _ in range(3)]
        ibm_get_plane(self.state, i, *out)
        return tuple(out)

    def set_probes(self, ijk):
        """Probe cells (n, 3) of (i, j, k)."""
        ibm_probes_set(self.state, ijk)

    def probe_sample(self, dst):
        """Cell-centred (u, v, w) of every probe into a device buffer (3 n values
        in the state's precision), asynchronous on the solver's stream."""
        ibm_probe_sample(self.state, dst)

    def save(self, path):
        ibm_save(self.state, path)

    def load(self, path):
        ibm_load(self.state, path)

    def time_stage(self, stage, nrep=10):
        return ibm_time_stage(self.state, STAGES[stage] if isinstance(stage, str) else stage, nrep)

    def close(self):
        if getattr(self, "state", None) is not None:
            ibm_destroy(self.state)
            self.state = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Several Solver members stepped together by one graph launch per step;
    batched: the members' explicit stages in one persistent launch."""

    def __init__(self, solvers, stream=None, batched=False):
        import torch
        self.solvers = list(solvers)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.handle = ibm_ensemble_create([s.state for s in self.solvers],
                                          ctypes.c_void_p(self.stream.cuda_stream), batched)

    def step(self, nsteps=1, dt=-1.0):
        _check(ibm_ensemble_step(self.handle, dt, nsteps), "ibm_ensemble_step")

    def close(self):
        if getattr(self, "handle", None) is not None:
            ibm_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Generator:
    """Learned inflow generator (ibm_gen_*): device buffers are torch tensors
    on the current CUDA device, the stream is torch's unless one is given."""

    def __init__(self, ny, nz, blocks=13, in_channels=6, batch=8, lr=1e-3, stream=None, stride=1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the generator needs a CUDA device")
        load()
        self.ny, self.nz, self.blocks, self.in_channels, self.batch = ny, nz, blocks, in_channels, batch
        self.stride = stride
        self.stream = stream if stream is not None else torch.cuda.Stream()
        cfg = ibm_gen_config(ny, nz, 128, blocks, in_channels, batch, lr, 0.0, 0.0, 0.0,
                             ctypes.c_void_p(self.stream.cuda_stream), stride)
        torch.cuda.synchronize()
        self.handle = ibm_gen_create(cfg)
        self.n_params = ibm_gen_param_count(self.handle)

    def _dev(self, a):
        import torch
        t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()
        torch.cuda.synchronize()
        return t

    def set_params(self, w):
        ibm_gen_set_params(self.handle, w)

    def params(self):
        out = np.empty(self.n_params)
        ibm_gen_get_params(self.handle, out)
        return out

    def grads(self):
        out = np.empty(self.n_params)
        ibm_gen_get_grads(self.handle, out)
        return out

    def set_norm(self, mean, std, rms):
        ibm_gen_set_norm(self.handle, mean, std, rms)

    def forward(self, q_t, q_prev):
        """q's [batch, ny, nz, 3] (host arrays or CUDA tensors) -> delta (host)."""
        import torch
        qt, qp = self._dev(q_t), self._dev(q_prev)
        out = torch.empty_like(qt)
        ibm_gen_forward(self.handle, qt.data_ptr(), qp.data_ptr(), out.data_ptr(), qt.shape[0])
        return out.cpu().numpy().astype(np.float64)

    def grad(self, q_t, q_prev, target):
        qt, qp, tg = self._dev(q_t), self._dev(q_prev), self._dev(target)
        return ibm_gen_grad(self.handle, qt.data_ptr(), qp.data_ptr(), tg.data_ptr(), qt.shape[0])

    def adam_step(self):
        ibm_gen_adam_step(self.handle)

    def train_step(self, planes, t_idx, with_loss=True):
        """planes: CUDA float32 tensor [n, 3, ny, nz]."""
        return ibm_gen_train_step(self.handle, planes.data_ptr(), planes.shape[0], t_idx, with_loss)

    def train_step_pushforward(self, planes, t_idx, with_loss=True):
        """The pushforward step: inputs from the network's own prediction of q_t."""
        return ibm_gen_train_step_pushforward(self.handle, planes.data_ptr(), planes.shape[0], t_idx, with_loss)

    def eval(self, planes, t_idx):
        return ibm_gen_eval(self.handle, planes.data_ptr(), planes.shape[0], t_idx)

    def set_lr(self, lr):
        ibm_gen_set_lr(self.handle, lr)

    def set_noise(self, std, seed=0):
        ibm_gen_set_noise(self.handle, std, seed)

    def set_relax(self, plane, lam):
        """plane: host [3, ny, nz] raw plane (e.g. the data's time mean)."""
        ibm_gen_set_relax(self.handle, plane, lam)

    def set_spectrum(self, power, lam):
        """power: host [3, ny, nz] target Fourier power of the normalised
        fluctuation about the relaxation plane (after set_relax)."""
        ibm_gen_set_spectrum(self.handle, power, lam)

    def time(self, what, nrep=10):
        return ibm_gen_time(self.handle, GEN_TIMINGS[what] if isinstance(what, str) else what, nrep)

    def rollout_init(self, plane_prev, plane_cur):
        self._init = (self._dev(plane_prev), self._dev(plane_cur))
        ibm_gen_rollout_init(self.handle, self._init[0].data_ptr(), self._init[1].data_ptr())

    def rollout(self, u, v, w, precision=IBM_FP32):
        ibm_gen_rollout(self.handle, u, v, w, precision)

    def emit(self, w, u, v, wv, precision=IBM_FP32):
        ibm_gen_emit(self.handle, w, u, v, wv, precision)

    def history(self):
        import torch
        qt = torch.empty((self.ny, self.nz, 3), dtype=torch.float32, device="cuda")
        qp = torch.empty_like(qt)
        ibm_gen_history(self.handle, qt.data_ptr(), qp.data_ptr())
        return qt.cpu().numpy().astype(np.float64), qp.cpu().numpy().astype(np.float64)

    def save(self, path):
        ibm_gen_save(self.handle, path)

    def load(self, path):
        ibm_gen_load(self.handle, path)

    def sync(self):
        ibm_gen_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            ibm_gen_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
