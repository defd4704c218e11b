"""Thin ctypes binding of the C ABI in ``include/dismech.h``.

Argument marshalling only: every step of the implicit DER solve runs in the
CUDA kernels of ``libdismech.so``.  Host arrays are numpy; device buffers
are torch CUDA tensors (their data pointers are passed with is_device=1).
The binding refuses to work without the compiled library: there is no CPU
fallback.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdismech.so")

DM_OK = 0
STATUS = {0: "DM_OK", 1: "DM_ERR_INVALID_ARG", 2: "DM_ERR_NOT_CONVERGED",
          3: "DM_ERR_NONFINITE", 4: "DM_ERR_DEGENERATE", 5: "DM_ERR_PENETRATION",
          6: "DM_ERR_CUDA", 7: "DM_ERR_OOM"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint8)


class SystemDesc(C.Structure):
    _fields_ = [("n_rods", C.c_int32), ("nodes_per_rod", _ip), ("x0", _dp), ("v0", _dp),
                ("theta0", _dp), ("theta_dot0", _dp), ("E", _dp), ("nu", _dp), ("rho", _dp),
                ("radius", _dp), ("n_joints", C.c_int32), ("joint_offsets", _ip),
                ("joint_members", _ip), ("fixed", _up), ("ground_mu", _dp), ("ground_kc", _dp),
                ("n_contact_groups", C.c_int32), ("contact_group_offsets", _ip),
                ("contact_group_rods", _ip)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("newton_tol", C.c_double), ("max_iter", C.c_int32),
                ("gravity", C.c_double * 3), ("damping", C.c_double), ("ground", C.c_int32),
                ("ground_z", C.c_double), ("delta", C.c_double), ("slip_nu", C.c_double),
                ("self_contact", C.c_int32), ("pair_kc", C.c_double), ("pair_mu", C.c_double),
                ("line_search", C.c_int32), ("stream", C.c_void_p), ("integrator", C.c_int32),
                ("long_rod_dofs", C.c_int32), ("predictor", C.c_int32)]

INTEGRATORS = {"be": 0, "midpoint": 1}
PREDICTORS = {"extrapolate": 0, "projected": 1}


class StepStats(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("iterations", _ip), ("residual", _dp),
                ("first_failed", C.c_int32), ("steps_done", C.c_int32),
                ("sum_iterations", C.c_int64), ("max_iterations", C.c_int32)]


NUM_KERNELS = 17


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * NUM_KERNELS), ("units", C.c_int64 * NUM_KERNELS),
                ("ms", C.c_double * NUM_KERNELS)]


TUNING_FIELDS = ("edge_threads", "stencil_threads", "stencil_per_thread", "rows_threads",
                 "solve_warps", "solve_blocks_per_sm", "limb_factor_warps", "limb_back_warps")


class Tuning(C.Structure):
    _fields_ = [(f, C.c_int32) for f in TUNING_FIELDS] + [("us_per_launch", C.c_double * 8)]


_lib = None


def load_library(path=LIB_PATH):
    """Loads ``libdismech.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdismech.so is missing: run __graft_entry__.build() "
                           "(no CPU fallback exists)")
    lib = C.CDLL(path)
    H = C.c_void_p
    lib.dm_create_system.argtypes = [C.POINTER(SystemDesc), C.POINTER(Params), C.POINTER(H)]
    lib.dm_create_system.restype = C.c_int
    lib.dm_destroy.argtypes = [H]
    lib.dm_destroy.restype = None
    lib.dm_set_natural_curvature.argtypes = [H, C.c_int32, C.c_int32, C.c_void_p, C.c_int32]
    lib.dm_set_natural_curvature.restype = C.c_int
    lib.dm_step.argtypes = [H, C.c_int32, C.POINTER(StepStats)]
    lib.dm_step.restype = C.c_int
    lib.dm_get_state.argtypes = [H, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32]
    lib.dm_get_state.restype = C.c_int
    lib.dm_set_state.argtypes = [H, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32]
    lib.dm_set_state.restype = C.c_int
    lib.dm_get_frames.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int32]
    lib.dm_get_frames.restype = C.c_int
    lib.dm_set_frames.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int32]
    lib.dm_set_frames.restype = C.c_int
    lib.dm_adjoint_frame_chain.argtypes = [H] + [C.c_void_p] * 8
    lib.dm_adjoint_frame_chain.restype = C.c_int
    lib.dm_state_size.argtypes = [H]
    lib.dm_state_size.restype = C.c_int64
    lib.dm_num_systems.argtypes = [H]
    lib.dm_num_systems.restype = C.c_int32
    lib.dm_num_stencils.argtypes = [H]
    lib.dm_num_stencils.restype = C.c_int64
    lib.dm_num_edges.argtypes = [H]
    lib.dm_num_edges.restype = C.c_int64
    lib.dm_autotune.argtypes = [H, C.c_int32, C.POINTER(Tuning)]
    lib.dm_autotune.restype = C.c_int
    lib.dm_set_tuning.argtypes = [H, C.POINTER(Tuning)]
    lib.dm_set_tuning.restype = C.c_int
    lib.dm_set_graphs.argtypes = [H, C.c_int32]
    lib.dm_set_graphs.restype = C.c_int
    lib.dm_set_fused_first.argtypes = [H, C.c_int32]
    lib.dm_set_fused_first.restype = C.c_int
    lib.dm_set_profiling.argtypes = [H, C.c_int32]
    lib.dm_set_profiling.restype = C.c_int
    lib.dm_get_profile.argtypes = [H, C.POINTER(Profile)]
    lib.dm_get_profile.restype = C.c_int
    lib.dm_kernel_name.argtypes = [C.c_int32]
    lib.dm_kernel_name.restype = C.c_char_p
    lib.dm_fp64_peak_gflops.argtypes = []
    lib.dm_fp64_peak_gflops.restype = C.c_double
    lib.dm_solve_band.argtypes = [C.c_int32, _ip, _ip, C.c_int64, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]
    lib.dm_solve_band.restype = C.c_int
    lib.dm_solve_band_partitioned.argtypes = lib.dm_solve_band.argtypes[:-1] + [C.c_int32,
                                                                                C.c_void_p]
    lib.dm_solve_band_partitioned.restype = C.c_int
    lib.dm_solve_band_noalloc.argtypes = lib.dm_solve_band.argtypes
    lib.dm_solve_band_noalloc.restype = C.c_int
    lib.dm_debug_copy.argtypes = [H, C.c_char_p, _dp, C.c_int64]
    lib.dm_debug_copy.restype = C.c_int
    lib.dm_gemm_bf16.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
    lib.dm_gemm_bf16.restype = C.c_int
    lib.dm_mlp_create.argtypes = [C.c_int32, C.c_int32, C.c_uint64, C.c_void_p,
                                  C.POINTER(C.c_void_p)]
    lib.dm_mlp_create.restype = C.c_int
    lib.dm_mlp_destroy.argtypes = [C.c_void_p]
    lib.dm_mlp_destroy.restype = None
    lib.dm_mlp_num_params.argtypes = []
    lib.dm_mlp_num_params.restype = C.c_int64
    lib.dm_mlp_get_params.argtypes = [C.c_void_p, C.POINTER(C.c_float)]
    lib.dm_mlp_get_params.restype = C.c_int
    lib.dm_mlp_set_params.argtypes = [C.c_void_p, C.POINTER(C.c_float)]
    lib.dm_mlp_set_params.restype = C.c_int
    lib.dm_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    lib.dm_mlp_forward.restype = C.c_int
    lib.dm_mlp_forward_async.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    lib.dm_mlp_forward_async.restype = C.c_int
    lib.dm_mlp_check.argtypes = [C.c_void_p]
    lib.dm_mlp_check.restype = C.c_int
    lib.dm_mlp_set_fused.argtypes = [C.c_void_p, C.c_int32]
    lib.dm_mlp_set_fused.restype = C.c_int
    lib.dm_mlp_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                      C.c_void_p, C.POINTER(C.c_double)]
    lib.dm_mlp_train_step.restype = C.c_int
    lib.dm_ws_enable.argtypes = [H]
    lib.dm_ws_enable.restype = C.c_int
    lib.dm_ws_num_segments.argtypes = [H]
    lib.dm_ws_num_segments.restype = C.c_int64
    lib.dm_ws_capture_features.argtypes = [H, C.c_void_p]
    lib.dm_ws_capture_features.restype = C.c_int
    lib.dm_ws_capture_targets.argtypes = [H, C.c_void_p]
    lib.dm_ws_capture_targets.restype = C.c_int
    lib.dm_ws_set_model.argtypes = [H, C.c_void_p, C.POINTER(C.c_float)]
    lib.dm_ws_set_model.restype = C.c_int
    lib.dm_ws_prepare_batch.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dm_ws_prepare_batch.restype = C.c_int
    lib.dm_ws_column_stats.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
    lib.dm_ws_column_stats.restype = C.c_int
    lib.dm_step_adjoint.argtypes = [H] + [C.c_void_p] * 6 + [C.c_int32]
    lib.dm_step_adjoint.restype = C.c_int
    lib.dm_contact_pairs.argtypes = [H]
    lib.dm_contact_pairs.restype = C.c_int64
    lib.dm_last_error.argtypes = []
    lib.dm_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class DismechError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def _check(code):
    if code != DM_OK:
        raise DismechError(code, _lib.dm_last_error().decode())


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def _dev_ptr(t):
    return C.c_void_p(t.data_ptr())


class System:
    """Batch of rod systems advanced by the GPU implicit DER step.

    ``desc``: dict with nodes_per_rod, x0, E, nu, rho, radius and optional
    v0, theta0, theta_dot0, joints (list of [(rod, node), ...]), fixed,
    ground_mu, ground_kc, contact_groups (list of lists of consecutive rods
    solved as one system so that they can touch each other).  ``params``:
    dt, tol, max_iter, g, eta, ground, ground_z, delta, nu_slip,
    self_contact, pair_kc, pair_mu, line_search, integrator ("be" or
    "midpoint"), long_rod_dofs (rods with at least this many DOFs use the
    partitioned band solve; 0 = 2048, negative = never), predictor
    ("extrapolate" or "projected": the guess rescaled to the committed edge
    lengths on single rods), stream.
    """

    def __init__(self, desc, params):
        lib = load_library()
        self._keep = []

        def arr(key, dtype, shape=None):
            v = desc.get(key)
            if v is None:
                return None
            a = np.ascontiguousarray(np.asarray(v, dtype=dtype))
            if shape is not None:
                a = a.reshape(shape)
            self._keep.append(a)
            return a

        npr = arr("nodes_per_rod", np.int32)
        d = SystemDesc()
        d.n_rods = len(npr)
        d.nodes_per_rod = _ptr(npr, C.c_int32)
        d.x0 = _ptr(arr("x0", np.float64, (-1,)), C.c_double)
        d.v0 = _ptr(arr("v0", np.float64, (-1,)), C.c_double)
        d.theta0 = _ptr(arr("theta0", np.float64), C.c_double)
        d.theta_dot0 = _ptr(arr("theta_dot0", np.float64), C.c_double)
        for k in ("E", "nu", "rho", "radius"):
            setattr(d, k, _ptr(arr(k, np.float64), C.c_double))
        joints = desc.get("joints") or []
        if joints:
            off = np.zeros(len(joints) + 1, np.int32)
            mem = []
            for j, grp in enumerate(joints):
                off[j + 1] = off[j] + len(grp)
                for (r, i) in grp:
                    mem += [r, i]
            mem = np.asarray(mem, np.int32)
            self._keep += [off, mem]
            d.n_joints = len(joints)
            d.joint_offsets = _ptr(off, C.c_int32)
            d.joint_members = _ptr(mem, C.c_int32)
        groups = desc.get("contact_groups") or []
        if groups:
            goff = np.zeros(len(groups) + 1, np.int32)
            goff[1:] = np.cumsum([len(g) for g in groups])
            grods = np.ascontiguousarray(np.concatenate([np.asarray(g, np.int32) for g in groups]),
                                         np.int32)
            self._keep += [goff, grods]
            d.n_contact_groups = len(groups)
            d.contact_group_offsets = _ptr(goff, C.c_int32)
            d.contact_group_rods = _ptr(grods, C.c_int32)
        d.fixed = _ptr(arr("fixed", np.uint8), C.c_uint8)
        d.ground_mu = _ptr(arr("ground_mu", np.float64), C.c_double)
        d.ground_kc = _ptr(arr("ground_kc", np.float64), C.c_double)
        p = Params()
        p.dt = params.get("dt", 1e-3)
        p.newton_tol = params.get("tol", 1e-10)
        p.max_iter = params.get("max_iter", 100)
        g = params.get("g", (0.0, 0.0, -9.81))
        for c in range(3):
            p.gravity[c] = g[c]
        p.damping = params.get("eta", 0.0)
        p.ground = int(bool(params.get("ground", False)))
        p.ground_z = params.get("ground_z", 0.0)
        p.delta = params.get("delta", 5e-4)
        p.slip_nu = params.get("nu_slip", 1e-3)
        p.self_contact = int(bool(params.get("self_contact", False)))
        p.pair_kc = params.get("pair_kc", 0.0)
        p.pair_mu = params.get("pair_mu", 0.0)
        p.line_search = int(bool(params.get("line_search", False)))
        p.stream = params.get("stream", None)
        integ = params.get("integrator", "be")
        if integ not in INTEGRATORS:
            raise ValueError("integrator must be one of %s" % sorted(INTEGRATORS))
        p.integrator = INTEGRATORS[integ]
        p.long_rod_dofs = int(params.get("long_rod_dofs", 0))
        pred = params.get("predictor", "extrapolate")
        if pred not in PREDICTORS:
            raise ValueError("predictor must be one of %s" % sorted(PREDICTORS))
        p.predictor = PREDICTORS[pred]
        h = C.c_void_p()
        _check(lib.dm_create_system(C.byref(d), C.byref(p), C.byref(h)))
        self._h = h
        self._lib = lib
        self.n_state = lib.dm_state_size(h)
        self.n_systems = lib.dm_num_systems(h)
        self.n_stencils = lib.dm_num_stencils(h)
        self.n_edges = lib.dm_num_edges(h)
        self.n_rods = d.n_rods
        self._npr = np.asarray(npr, np.int64)
        self.dt = float(p.dt)
        fx = desc.get("fixed")
        self._fixed = (np.zeros(int(np.sum(4 * self._npr - 1)), bool) if fx is None
                       else np.asarray(fx).astype(bool).reshape(-1))
        self.stats = StepStats()
        self._iters = np.zeros(self.n_systems, np.int32)
        self._res = np.zeros(self.n_systems, np.float64)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1, stats=True):
        st = self.stats
        if stats:
            st.capacity = self.n_systems
            st.iterations = _ptr(self._iters, C.c_int32)
            st.residual = _ptr(self._res, C.c_double)
        else:
            st.capacity = 0
            st.iterations = None
            st.residual = None
        _check(self._lib.dm_step(self._h, nsteps, C.byref(st)))
        return st

    @property
    def iterations(self):
        return self._iters.copy()

    @property
    def residual(self):
        return self._res.copy()

    def set_natural_curvature(self, rod_begin, rod_end, kbar):
        if hasattr(kbar, "data_ptr"):
            _check(self._lib.dm_set_natural_curvature(self._h, rod_begin, rod_end,
                                                      _dev_ptr(kbar), 1))
        else:
            k = np.ascontiguousarray(np.asarray(kbar, np.float64).reshape(-1))
            _check(self._lib.dm_set_natural_curvature(self._h, rod_begin, rod_end,
                                                      k.ctypes.data_as(C.c_void_p), 0))

    def get_state(self, q=None, qdot=None):
        """(q, qdot) in the per-rod layout of Eq. 1.  Into torch CUDA tensors
        when given; into caller-owned host arrays (numpy float64, e.g. views
        of pinned memory, which copy fastest) when given; otherwise into new
        numpy arrays."""
        if q is not None and hasattr(q, "data_ptr"):
            _check(self._lib.dm_get_state(self._h, _dev_ptr(q),
                                          _dev_ptr(qdot) if qdot is not None else None,
                                          self.n_state, 1))
            return q, qdot
        q = np.zeros(self.n_state) if q is None else q
        v = np.zeros(self.n_state) if qdot is None else qdot
        for a in (q, v):
            if (a.dtype != np.float64 or not a.flags.c_contiguous or a.size < self.n_state):
                raise ValueError("host state buffers must be contiguous float64 arrays of "
                                 "at least %d entries" % self.n_state)
        _check(self._lib.dm_get_state(self._h, q.ctypes.data_as(C.c_void_p),
                                      v.ctypes.data_as(C.c_void_p), q.size, 0))
        return q, v

    def set_state(self, q, qdot):
        if hasattr(q, "data_ptr"):
            _check(self._lib.dm_set_state(self._h, _dev_ptr(q), _dev_ptr(qdot),
                                          self.n_state, 1))
            return
        q = np.ascontiguousarray(np.asarray(q, np.float64))
        v = np.ascontiguousarray(np.asarray(qdot, np.float64))
        _check(self._lib.dm_set_state(self._h, q.ctypes.data_as(C.c_void_p),
                                      v.ctypes.data_as(C.c_void_p), len(q), 0))

    def autotune(self, steps=2):
        """Chooses the launch shapes of the edge, stencil, row, rod-solve
        and limb-solve kernels by timing candidates on this system from its
        current state (which is left unchanged); returns the choice and the
        measured microseconds per launch of the chosen shapes."""
        t = Tuning()
        _check(self._lib.dm_autotune(self._h, int(steps), C.byref(t)))
        out = {f: int(getattr(t, f)) for f in TUNING_FIELDS}
        out["us_per_launch"] = dict(zip(("edge", "stencil", "rows", "rod_solve",
                                         "limb_solve_factor", "limb_solve_back"),
                                        [round(float(x), 2) for x in t.us_per_launch[:6]]))
        return out

    def set_tuning(self, tuning):
        """Applies launch shapes returned by autotune() (a dict with the
        Tuning fields; us_per_launch is ignored) without timing anything."""
        t = Tuning()
        for f in TUNING_FIELDS:
            setattr(t, f, int(tuning[f]))
        _check(self._lib.dm_set_tuning(self._h, C.byref(t)))

    def set_graphs(self, enable=True):
        """Newton rounds as one CUDA graph per step (default) or host-driven."""
        _check(self._lib.dm_set_graphs(self._h, int(bool(enable))))

    def set_fused_first(self, enable=True):
        """First round of a step by the fused passes (default) or the split ones."""
        _check(self._lib.dm_set_fused_first(self._h, int(bool(enable))))

    def set_profiling(self, enable=True):
        _check(self._lib.dm_set_profiling(self._h, int(bool(enable))))

    def get_profile(self):
        """{kernel name: (launches, units, ms)} for kernels that ran."""
        p = Profile()
        _check(self._lib.dm_get_profile(self._h, C.byref(p)))
        out = {}
        for k in range(NUM_KERNELS):
            name = self._lib.dm_kernel_name(k).decode()
            if name and p.launches[k]:
                out[name] = (int(p.launches[k]), int(p.units[k]), float(p.ms[k]))
        return out

    def debug_copy(self, name, n):
        out = np.zeros(int(n))
        _check(self._lib.dm_debug_copy(self._h, name.encode(), _ptr(out, C.c_double), len(out)))
        return out

    def get_frames(self, d1=None, beta=None):
        """(d1 [edges, 3], beta [stencils]): into torch CUDA tensors when
        given (no synchronisation), else new numpy arrays."""
        if d1 is not None and hasattr(d1, "data_ptr"):
            _check(self._lib.dm_get_frames(self._h, _dev_ptr(d1), _dev_ptr(beta), 1))
            return d1, beta
        d1 = np.zeros((self.n_edges, 3))
        beta = np.zeros(self.n_stencils)
        _check(self._lib.dm_get_frames(self._h, d1.ctypes.data_as(C.c_void_p),
                                       beta.ctypes.data_as(C.c_void_p), 0))
        return d1, beta

    def set_frames(self, d1, beta):
        if hasattr(d1, "data_ptr"):
            _check(self._lib.dm_set_frames(self._h, _dev_ptr(d1), _dev_ptr(beta), 1))
            return
        d1 = np.ascontiguousarray(np.asarray(d1, np.float64))
        beta = np.ascontiguousarray(np.asarray(beta, np.float64))
        _check(self._lib.dm_set_frames(self._h, d1.ctypes.data_as(C.c_void_p),
                                       beta.ctypes.data_as(C.c_void_p), 0))

    def adjoint_frame_chain(self, q_prev, q, q_next, gq, gv, gv0, phibar, gq0):
        """One step of the rollout adjoint's frame chain (torch CUDA
        float64 tensors; phibar and gq0 updated in place)."""
        p = lambda t: _dev_ptr(t) if t is not None else None
        _check(self._lib.dm_adjoint_frame_chain(self._h, p(q_prev), p(q), p(q_next), p(gq),
                                                p(gv), p(gv0), p(phibar), p(gq0)))


    def step_adjoint(self, q_next, gq, gv):
        """Adjoint of the step from the current state (step n) to q_next:
        returns (dL/dkappabar [slots, 2], dL/dq_n, dL/dqdot_n) for the loss
        gradients gq = dL/dq_{n+1}, gv = dL/dqdot_{n+1} (host numpy, or
        torch CUDA float64 tensors, returned as such)."""
        if hasattr(q_next, "data_ptr"):
            import torch
            nslots = int(np.sum(self._npr - 2))
            gk = torch.zeros((max(nslots, 1), 2), dtype=torch.float64, device=q_next.device)
            gq0 = torch.empty_like(q_next)
            gv0 = torch.empty_like(q_next)
            _check(self._lib.dm_step_adjoint(self._h, _dev_ptr(q_next), _dev_ptr(gq),
                                             _dev_ptr(gv), _dev_ptr(gk), _dev_ptr(gq0),
                                             _dev_ptr(gv0), 1))
            return gk[:nslots], gq0, gv0
        f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64))
        q_next, gq, gv = f(q_next), f(gq), f(gv)
        nslots = int(np.sum(self._npr - 2))
        gk = np.zeros((max(nslots, 1), 2))
        gq0 = np.zeros(self.n_state)
        gv0 = np.zeros(self.n_state)
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        _check(self._lib.dm_step_adjoint(self._h, ptr(q_next), ptr(gq), ptr(gv), ptr(gk),
                                         ptr(gq0), ptr(gv0), 0))
        return gk[:nslots], gq0, gv0

    def fixed_mask(self):
        """Fixed-DOF mask in the dm_get_state layout (from the descriptor)."""
        return self._fixed.copy()

    def contact_pairs(self):
        """Edge pairs in contact at the last evaluated Newton iterate."""
        return int(self._lib.dm_contact_pairs(self._h))

    # ----- learned warm start -------------------------------------------
    def ws_enable(self):
        """Builds the warm-start segment tables; returns their number."""
        _check(self._lib.dm_ws_enable(self._h))
        return int(self._lib.dm_ws_num_segments(self._h))

    def ws_capture_features(self, feat):
        """Raw features [S, 64] (torch CUDA float32) of the committed state;
        asynchronous on the system's stream."""
        _check(self._lib.dm_ws_capture_features(self._h, _dev_ptr(feat)))
        return feat

    def ws_capture_targets(self, tgt):
        """Targets [S, 4] (torch CUDA float32) of the step just taken,
        relative to the guess remembered by ws_capture_features."""
        _check(self._lib.dm_ws_capture_targets(self._h, _dev_ptr(tgt)))
        return tgt

    def ws_set_model(self, mlp, norm=None):
        """Attaches a trained MLP (out_dim 4) with its normalisation (132
        floats: input mean, input std, output scale); None detaches."""
        if mlp is None:
            _check(self._lib.dm_ws_set_model(self._h, None, None))
            self._ws_model = None
            return
        n = np.ascontiguousarray(np.asarray(norm, np.float32))
        if n.size != 132:
            raise ValueError("norm must hold 132 floats")
        _check(self._lib.dm_ws_set_model(self._h, mlp._h, n.ctypes.data_as(C.POINTER(C.c_float))))
        self._ws_model = mlp  # keeps the network alive while attached


def ws_prepare_batch(feat, tgt, idx, norm, X, Y, stream=None):
    """X [M, 64] bf16 = normalised feat[idx], Y [M, 4] f32 = tgt[idx] /
    output scale (torch CUDA tensors; norm a float32 CUDA tensor [132])."""
    lib = load_library()
    _check(lib.dm_ws_prepare_batch(_dev_ptr(feat), _dev_ptr(tgt), _dev_ptr(idx), idx.numel(),
                                   _dev_ptr(norm), _dev_ptr(X), _dev_ptr(Y), stream))
    return X, Y


def ws_column_stats(data, stats, stream=None):
    """stats [2, cols] = column means and standard deviations of data
    [rows, cols] (torch CUDA float32)."""
    lib = load_library()
    rows, cols = data.shape
    _check(lib.dm_ws_column_stats(_dev_ptr(data), rows, cols, _dev_ptr(stats), stream))
    return stats


def solve_band(sys_dof0, sys_ndof, band, rhs, x, stream=None):
    """J x = rhs for a batch of symmetric banded rod systems (half bandwidth
    10) on the GPU.  band [11, ntot], rhs and x [ntot]: torch CUDA float64
    tensors; sys_dof0/sys_ndof: host integer sequences."""
    lib = load_library()
    d0 = np.ascontiguousarray(np.asarray(sys_dof0, np.int32))
    nd = np.ascontiguousarray(np.asarray(sys_ndof, np.int32))
    _check(lib.dm_solve_band(len(d0), _ptr(d0, C.c_int32), _ptr(nd, C.c_int32), x.numel(),
                             _dev_ptr(band), _dev_ptr(rhs), _dev_ptr(x), stream))
    return x


def solve_band_partitioned(sys_dof0, sys_ndof, band, rhs, x, part_rows=0, stream=None):
    """solve_band for long systems: interiors of part_rows - 10 rows factored
    in parallel, a block-tridiagonal Schur system on the 10-row separators
    (part_rows 0 = 512)."""
    lib = load_library()
    d0 = np.ascontiguousarray(np.asarray(sys_dof0, np.int32))
    nd = np.ascontiguousarray(np.asarray(sys_ndof, np.int32))
    _check(lib.dm_solve_band_partitioned(len(d0), _ptr(d0, C.c_int32), _ptr(nd, C.c_int32),
                                         x.numel(), _dev_ptr(band), _dev_ptr(rhs), _dev_ptr(x),
                                         int(part_rows), stream))
    return x


NOALLOC_MAX_SYSTEMS = 2048
NOALLOC_MAX_DOFS = 32768


def solve_band_noalloc(sys_dof0, sys_ndof, band, rhs, x, stream=None):
    """solve_band without device allocation, for callers that cannot allocate
    (real-time loops that cannot take cudaMalloc's device-wide
    synchronisation, processes whose device memory belongs to another
    allocator).  The scratch is one fixed library array of at most
    NOALLOC_MAX_SYSTEMS systems / NOALLOC_MAX_DOFS DOFs; calls that overlap
    on the GPU race on it."""
    lib = load_library()
    d0 = np.ascontiguousarray(np.asarray(sys_dof0, np.int32))
    nd = np.ascontiguousarray(np.asarray(sys_ndof, np.int32))
    _check(lib.dm_solve_band_noalloc(len(d0), _ptr(d0, C.c_int32), _ptr(nd, C.c_int32),
                                     x.numel(), _dev_ptr(band), _dev_ptr(rhs), _dev_ptr(x),
                                     stream))
    return x


def gemm_bf16(A, B, bias, C, relu=False, stream=None):
    """C = act(A B^T + bias) on the tcgen05 tensor cores (torch CUDA tensors:
    A [M, K] and B [N, K] bfloat16, bias [N] float32 or None, C [M, N]
    bfloat16 or float32)."""
    lib = load_library()
    M, K = A.shape
    N = B.shape[0]
    out_f32 = 1 if C.dtype.itemsize == 4 else 0
    _check(lib.dm_gemm_bf16(M, N, K, _dev_ptr(A), _dev_ptr(B),
                            _dev_ptr(bias) if bias is not None else None, _dev_ptr(C),
                            int(bool(relu)), out_f32, stream))
    return C


class MLP:
    """The warm-start network of the library (tensor-core training and
    inference).  Device buffers are torch CUDA tensors."""

    def __init__(self, in_dim, out_dim, seed=0, stream=None):
        self._lib = load_library()
        h = C.c_void_p()
        _check(self._lib.dm_mlp_create(in_dim, out_dim, seed, stream, C.byref(h)))
        self._h = h
        self.in_dim, self.out_dim = in_dim, out_dim
        self.n_params = int(self._lib.dm_mlp_num_params())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        _check(self._lib.dm_mlp_get_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, np.float32))
        _check(self._lib.dm_mlp_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def forward(self, X, Y):
        _check(self._lib.dm_mlp_forward(self._h, _dev_ptr(X), _dev_ptr(Y), X.shape[0]))
        return Y

    def forward_async(self, X, Y):
        """Enqueues inference on the network's stream without synchronising;
        check() reports a failure of it."""
        _check(self._lib.dm_mlp_forward_async(self._h, _dev_ptr(X), _dev_ptr(Y), X.shape[0]))
        return Y

    def check(self):
        _check(self._lib.dm_mlp_check(self._h))

    def set_fused(self, enable=True):
        """Inference by the fused 4-layer kernel (default) or a GEMM per layer."""
        _check(self._lib.dm_mlp_set_fused(self._h, int(bool(enable))))

    def train_step(self, X, Y, lr, grads=None):
        loss = C.c_double()
        _check(self._lib.dm_mlp_train_step(self._h, _dev_ptr(X), _dev_ptr(Y), X.shape[0],
                                           float(lr), _dev_ptr(grads) if grads is not None
                                           else None, C.byref(loss)))
        return loss.value


def fp64_peak_gflops():
    """Measured FP64 FMA throughput of the current device (GFLOP/s)."""
    return float(load_library().dm_fp64_peak_gflops())


def ensure_built():
    """Compiles the library if it is missing (used by tests and tools)."""
    if not os.path.exists(LIB_PATH):
        _build.build()
    return load_library()
