"""ctypes binding of the C ABI in include/agis.h (argument marshalling only).

Every computation happens in libagis.so; this module only converts NumPy arrays or
torch tensors (host or CUDA) to pointers and the C structs to Python values.  Importing it
raises if the library is missing, so nothing silently falls back to a CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libagis.so")

AGIS_OK = 0
ERRORS = {-1: "AGIS_E_INVALID", -2: "AGIS_E_CUDA", -3: "AGIS_E_OOM", -4: "AGIS_E_TIMEOUT", -5: "AGIS_E_NONFINITE"}
N_CCD, N_ROW = 62, 7

# every symbol declared in include/agis.h
ABI_VERSION = 8  # AGIS_ABI_VERSION of include/agis.h
EXPORTS = (
    "agis_default_config", "agis_init", "agis_source_update", "agis_attitude_update", "agis_calibration_update",
    "agis_frame_rotate", "agis_iterate", "agis_evaluate", "agis_get_sources", "agis_get_attitude",
    "agis_get_calibration", "agis_set_sources", "agis_set_attitude", "agis_set_calibration", "agis_get_residuals",
    "agis_get_source_stats", "agis_get_sizes", "agis_get_kernel_times", "agis_destroy", "agis_last_error",
    "agis_abi_version", "agis_source_update_static", "agis_mlp_pack", "agis_mlp_forward", "agis_mlp_loss_grad",
    "agis_mlp_adam", "agis_proposal_targets", "agis_set_proposal", "agis_get_proposal_features",
    "agis_copy_sources_device", "agis_set_asi", "agis_asi_estimate", "agis_autotune", "agis_get_tuning",
    "agis_set_tuning", "agis_set_attnoise", "agis_get_attnoise", "agis_exchange_size", "agis_accumulate",
    "agis_get_exchange", "agis_set_exchange", "agis_solve_exchange",
)
X_ATTITUDE, X_CALIBRATION, X_FRAME = 0, 1, 2  # AGIS_X_* of include/agis.h
KNOBS = ("obs_pass", "src_batch", "mix_sums", "mix_solve5", "att_accum", "cal_accum")  # AGIS_KNOB_* order
STATIC_MAX_OBS = 16384
MLP_N_IN, MLP_N_OUT, MLP_N_PARAMS, MLP_PACKED_BYTES = 22, 5, 5957, 16032


class Geometry(C.Structure):
    _fields_ = [
        ("gamma_c", C.c_double), ("focal_length", C.c_double), ("p_ac", C.c_double), ("mu_c", C.c_double),
        ("eta0", C.c_double * N_CCD), ("x_fpa", C.c_double * N_CCD), ("x_centre", C.c_double * 2),
        ("ccd_row", C.c_int32 * N_CCD), ("orb_L0", C.c_double), ("obliquity", C.c_double),
        ("au_light_s", C.c_double), ("year_s", C.c_double), ("t_ep_ns", C.c_int64), ("t_fr_ns", C.c_int64),
        ("knot0_ns", C.c_int64), ("knot_dt_ns", C.c_int64), ("cal_t0_ns", C.c_int64), ("cal_dt_ns", C.c_int64),
        ("n_coef", C.c_int32), ("n_cal_days", C.c_int32),
    ]


class Config(C.Structure):
    _fields_ = [
        ("robust", C.c_int32), ("n_rounds", C.c_int32), ("n_eps", C.c_int32), ("weight_fn", C.c_int32),
        ("lambda_att", C.c_double), ("rhs_norm_term", C.c_int32), ("seg_len", C.c_int32),
        ("seg_overlap", C.c_int32), ("frame_each_iter", C.c_int32), ("block_mask", C.c_int32),
        ("use_graph", C.c_int32), ("pivot_tol", C.c_double), ("max_obs_per_source", C.c_int32),
        ("precision", C.c_int32), ("refresh_every", C.c_int32), ("block_order", C.c_int32),
        ("cal_model", C.c_int32), ("n_gate", C.c_int32), ("cal_j_per_k", C.c_int32), ("cal_col_bin", C.c_int32),
    ]


class Obs(C.Structure):
    _fields_ = [("t_ns", C.c_void_p), ("src", C.c_void_p), ("ccd", C.c_void_p), ("fov", C.c_void_p),
                ("kind", C.c_void_p), ("sigma", C.c_void_p), ("mu", C.c_void_p), ("gate", C.c_void_p)]


class BlockStats(C.Structure):
    _fields_ = [("chi2", C.c_double), ("q_sum", C.c_double), ("nu_sum", C.c_int64), ("n_out", C.c_int64),
                ("rank_defect", C.c_int64), ("d_rms", C.c_double * 5), ("elapsed_ms", C.c_double),
                ("pass_ms", C.c_double), ("full_eval", C.c_int32), ("reserved_", C.c_int32)]

    def as_dict(self):
        return dict(chi2=self.chi2, q_sum=self.q_sum, nu_sum=self.nu_sum, n_out=self.n_out,
                    rank_defect=self.rank_defect, d_rms=list(self.d_rms), elapsed_ms=self.elapsed_ms,
                    pass_ms=self.pass_ms, full_eval=self.full_eval)


class TuneEntry(C.Structure):
    _fields_ = [("knob", C.c_int32), ("a", C.c_int32), ("b", C.c_int32), ("n_tried", C.c_int32),
                ("best_ms", C.c_double), ("default_ms", C.c_double)]


class IterStats(C.Structure):
    _fields_ = [("s", BlockStats), ("a", BlockStats), ("c", BlockStats), ("frame", C.c_double * 6),
                ("elapsed_ms", C.c_double), ("proposal", C.c_int32), ("asi_n", C.c_int32),
                ("asi_lambda", C.c_double), ("asi_factor", C.c_double)]


_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1112_4139_gb300._build.build()")
        lib = C.CDLL(LIB_PATH)
        V, I, P = C.c_void_p, C.c_int, C.c_void_p
        lib.agis_default_config.argtypes = [C.POINTER(Config)]
        lib.agis_default_config.restype = None
        lib.agis_init.argtypes = [C.POINTER(Geometry), C.POINTER(Config), C.POINTER(Obs), C.c_int64, P, P, C.c_int32,
                                  P, C.c_int32, P, C.c_int32, P, C.POINTER(V)]
        lib.agis_init.restype = I
        for f in ("agis_source_update", "agis_attitude_update", "agis_calibration_update"):
            getattr(lib, f).argtypes = [V, C.POINTER(BlockStats)]
            getattr(lib, f).restype = I
        lib.agis_frame_rotate.argtypes = [V, P, C.c_int32, P]
        lib.agis_frame_rotate.restype = I
        lib.agis_iterate.argtypes = [V, C.c_int32, P, C.POINTER(C.c_int32)]
        lib.agis_iterate.restype = I
        for f in ("agis_evaluate", "agis_get_sources", "agis_get_attitude", "agis_get_calibration",
                  "agis_set_sources", "agis_set_attitude", "agis_set_calibration"):
            getattr(lib, f).argtypes = [V, P]
            getattr(lib, f).restype = I
        lib.agis_get_residuals.argtypes = [V, P, P]
        lib.agis_get_residuals.restype = I
        lib.agis_get_source_stats.argtypes = [V, P, P]
        lib.agis_get_source_stats.restype = I
        lib.agis_get_sizes.argtypes = [V, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32)]
        lib.agis_get_sizes.restype = I
        lib.agis_get_kernel_times.argtypes = [V, P]
        lib.agis_get_kernel_times.restype = I
        lib.agis_destroy.argtypes = [V]
        lib.agis_destroy.restype = None
        lib.agis_last_error.argtypes = [V]
        lib.agis_last_error.restype = C.c_char_p
        lib.agis_abi_version.restype = I
        lib.agis_source_update_static.argtypes = [C.POINTER(Geometry), C.POINTER(Config), C.POINTER(Obs), C.c_int64,
                                                  P, C.c_int32, P, P, P, P, P, C.c_int32, P]
        lib.agis_source_update_static.restype = I
        lib.agis_mlp_pack.argtypes = [P, P, V]
        lib.agis_mlp_forward.argtypes = [P, P, C.c_int32, P, V]
        lib.agis_mlp_loss_grad.argtypes = [P, P, P, P, C.c_int32, P, P, V]
        lib.agis_mlp_adam.argtypes = [P, P, P, P, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float, V]
        lib.agis_proposal_targets.argtypes = [P, P, P, C.c_int32, P, V]
        lib.agis_set_proposal.argtypes = [V, P, C.c_int32]
        lib.agis_get_proposal_features.argtypes = [V, P, P]
        lib.agis_copy_sources_device.argtypes = [V, P]
        lib.agis_set_asi.argtypes = [V, C.c_int32, C.c_double]
        lib.agis_asi_estimate.argtypes = [P, P, C.c_int32, C.c_int32, C.c_double, P, P, V]
        lib.agis_autotune.argtypes = [V, C.c_int32, C.POINTER(C.c_int32), P]
        lib.agis_get_tuning.argtypes = [V, P]
        lib.agis_set_tuning.argtypes = [V, P, C.c_int32]
        lib.agis_set_attnoise.argtypes = [V, C.c_int64]
        lib.agis_get_attnoise.argtypes = [V, P, C.POINTER(C.c_int32)]
        lib.agis_exchange_size.argtypes = [V, C.c_int32, C.POINTER(C.c_int64)]
        lib.agis_exchange_size.restype = I
        lib.agis_accumulate.argtypes = [V, C.c_int32]
        lib.agis_accumulate.restype = I
        for f in ("agis_get_exchange", "agis_set_exchange"):
            getattr(lib, f).argtypes = [V, C.c_int32, P]
            getattr(lib, f).restype = I
        lib.agis_solve_exchange.argtypes = [V, C.c_int32, C.POINTER(BlockStats), P]
        lib.agis_solve_exchange.restype = I
        for f in ("agis_mlp_pack", "agis_mlp_forward", "agis_mlp_loss_grad", "agis_mlp_adam", "agis_proposal_targets",
                  "agis_set_proposal", "agis_get_proposal_features", "agis_copy_sources_device", "agis_set_asi",
                  "agis_asi_estimate", "agis_autotune", "agis_get_tuning", "agis_set_tuning", "agis_set_attnoise",
                  "agis_get_attnoise"):
            getattr(lib, f).restype = I
        if lib.agis_abi_version() != ABI_VERSION:
            raise RuntimeError(f"libagis.so has ABI {lib.agis_abi_version()}, this binding {ABI_VERSION}: rebuild")
        _lib = lib
    return _lib


class AgisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(a):
    """Pointer of a NumPy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def geometry_from_dict(g: dict) -> Geometry:
    G = Geometry()
    G.gamma_c, G.focal_length, G.p_ac, G.mu_c = g["gamma_c"], g["focal_length"], g["p_ac"], g["mu_c"]
    G.eta0[:] = list(map(float, g["eta0"]))
    G.x_fpa[:] = list(map(float, g["x_fpa"]))
    G.x_centre[:] = list(map(float, g["x_centre"]))
    G.ccd_row[:] = list(map(int, g["ccd_row"]))
    G.orb_L0, G.obliquity, G.au_light_s, G.year_s = g["orb_L0"], g["obliquity"], g["au_light_s"], g["year_s"]
    G.t_ep_ns, G.t_fr_ns, G.knot0_ns, G.knot_dt_ns = g["t_ep_ns"], g["t_fr_ns"], g["knot0_ns"], g["knot_dt_ns"]
    G.cal_t0_ns, G.cal_dt_ns = g["cal_t0_ns"], g["cal_dt_ns"]
    G.n_coef, G.n_cal_days = g["n_coef"], g["n_cal_days"]
    return G


def default_config(**over) -> Config:
    cfg = Config()
    load().agis_default_config(C.byref(cfg))
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


class Agis:
    """One context of the GPU library (create, run blocks, read back, destroy)."""

    def __init__(self, geometry: dict, cfg: Config, obs: dict, src0, att0, cal0, src_ref=None, stream=None):
        lib = load()
        self._lib = lib
        self._keep = (obs, src0, att0, cal0, src_ref)
        o = Obs(*(_ptr(obs.get(k)) for k in ("t_ns", "src", "ccd", "fov", "kind", "sigma", "mu", "gate")))
        self.n_obs = int(obs["t_ns"].shape[0])
        self.n_src = int(src0.shape[0])
        self.n_coef = int(att0.shape[0])
        self.n_cal = int(cal0.shape[0])
        G = geometry_from_dict(geometry)
        ctx = C.c_void_p()
        s = C.c_void_p(stream) if stream is not None else None
        rc = lib.agis_init(C.byref(G), C.byref(cfg), C.byref(o), self.n_obs, _ptr(src0), _ptr(src_ref), self.n_src,
                           _ptr(att0), self.n_coef, _ptr(cal0), self.n_cal, s, C.byref(ctx))
        if rc != AGIS_OK:
            raise AgisError(rc, lib.agis_last_error(None).decode())
        self.ctx = ctx
        self._keep = None

    def _check(self, rc):
        if rc != AGIS_OK:
            raise AgisError(rc, self._lib.agis_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.agis_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # blocks
    def source_update(self):
        st = BlockStats()
        self._check(self._lib.agis_source_update(self.ctx, C.byref(st)))
        return st.as_dict()

    def attitude_update(self):
        st = BlockStats()
        self._check(self._lib.agis_attitude_update(self.ctx, C.byref(st)))
        return st.as_dict()

    def calibration_update(self):
        st = BlockStats()
        self._check(self._lib.agis_calibration_update(self.ctx, C.byref(st)))
        return st.as_dict()

    def frame_rotate(self, subset=None):
        eo = np.zeros(6)
        sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
        self._check(self._lib.agis_frame_rotate(self.ctx, _ptr(sub), 0 if sub is None else sub.size, _ptr(eo)))
        return eo

    def iterate(self, n_iter):
        arr = (IterStats * max(1, n_iter))()
        done = C.c_int32(0)
        self._check(self._lib.agis_iterate(self.ctx, n_iter, C.cast(arr, C.c_void_p), C.byref(done)))
        return [dict(s=arr[k].s.as_dict(), a=arr[k].a.as_dict(), c=arr[k].c.as_dict(), frame=list(arr[k].frame),
                     elapsed_ms=arr[k].elapsed_ms, proposal=arr[k].proposal, asi_n=arr[k].asi_n,
                     asi_lambda=arr[k].asi_lambda, asi_factor=arr[k].asi_factor) for k in range(done.value)]

    # read-back
    def evaluate(self, out=None):
        out = np.empty(self.n_obs) if out is None else out
        self._check(self._lib.agis_evaluate(self.ctx, _ptr(out)))
        return out

    def sources(self, out=None):
        out = np.empty((self.n_src, 5)) if out is None else out
        self._check(self._lib.agis_get_sources(self.ctx, _ptr(out)))
        return out

    def attitude(self, out=None):
        out = np.empty((self.n_coef, 4)) if out is None else out
        self._check(self._lib.agis_get_attitude(self.ctx, _ptr(out)))
        return out

    def calibration(self, out=None):
        out = np.empty(self.n_cal) if out is None else out
        self._check(self._lib.agis_get_calibration(self.ctx, _ptr(out)))
        return out

    def set_state(self, src=None, att=None, cal=None):
        if src is not None:
            self._check(self._lib.agis_set_sources(self.ctx, _ptr(np.ascontiguousarray(src, dtype=np.float64))))
        if att is not None:
            self._check(self._lib.agis_set_attitude(self.ctx, _ptr(np.ascontiguousarray(att, dtype=np.float64))))
        if cal is not None:
            self._check(self._lib.agis_set_calibration(self.ctx, _ptr(np.ascontiguousarray(cal, dtype=np.float64))))

    def residuals(self):
        R, W = np.empty(self.n_obs), np.empty(self.n_obs)
        self._check(self._lib.agis_get_residuals(self.ctx, _ptr(R), _ptr(W)))
        return R, W

    def source_stats(self):
        st = np.empty((5, self.n_src))
        cov = np.empty((self.n_src, 5, 5))
        self._check(self._lib.agis_get_source_stats(self.ctx, _ptr(st), _ptr(cov)))
        return dict(eps2=st[0], Q=st[1], nu=st[2], n_out=st[3], D=st[4], cov=cov)

    def kernel_times(self):
        ms = np.zeros(5)
        self._check(self._lib.agis_get_kernel_times(self.ctx, _ptr(ms)))
        return ms

    # learned proposal
    def set_proposal(self, params, every=5):
        """Enable the proposal with FP32 parameters (host array or device tensor); None disables."""
        if params is None:
            self._check(self._lib.agis_set_proposal(self.ctx, None, 0))
            return
        if isinstance(params, np.ndarray):
            params = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._lib.agis_set_proposal(self.ctx, _ptr(params), int(every)))

    def proposal_features(self, X, sigma):
        """Features (n_src x 22 FP32) and scales (n_src FP64) into device tensors."""
        self._check(self._lib.agis_get_proposal_features(self.ctx, _ptr(X), _ptr(sigma)))

    def copy_sources_device(self, out):
        self._check(self._lib.agis_copy_sources_device(self.ctx, _ptr(out)))

    # launch-shape autotuner
    def autotune(self, max_iter=16):
        """Run up to max_iter iterations rating candidate launch shapes; returns (iterations
        run, {knob: dict(a, b, n_tried, best_ms, default_ms)})."""
        arr = (TuneEntry * 6)()
        done = C.c_int32(0)
        self._check(self._lib.agis_autotune(self.ctx, int(max_iter), C.byref(done), C.cast(arr, C.c_void_p)))
        return done.value, _tune_dict(arr)

    def tuning(self):
        arr = (TuneEntry * 6)()
        self._check(self._lib.agis_get_tuning(self.ctx, C.cast(arr, C.c_void_p)))
        return _tune_dict(arr)

    def set_tuning(self, shapes):
        """shapes: {knob name: (a, b)}."""
        arr = (TuneEntry * max(1, len(shapes)))()
        for i, (name, (a, b)) in enumerate(shapes.items()):
            arr[i].knob, arr[i].a, arr[i].b = KNOBS.index(name), int(a), int(b)
        self._check(self._lib.agis_set_tuning(self.ctx, C.cast(arr, C.c_void_p), len(shapes)))

    # accelerated simple iteration
    def set_asi(self, stride=16, lambda_max=0.9):
        """Extrapolate the source update of each iteration by 1/(1 - lambda), lambda from the
        parallax updates of every stride-th source; stride 0 disables."""
        self._check(self._lib.agis_set_asi(self.ctx, int(stride), float(lambda_max)))

    # excess attitude noise
    def set_attnoise(self, bucket_ns):
        """Estimate the excess attitude noise on buckets of bucket_ns from knot0_ns; 0 disables."""
        self._check(self._lib.agis_set_attnoise(self.ctx, int(bucket_ns)))

    def attnoise(self):
        """eps_a^2 [3, n_buckets] (AL, AC preceding field, AC following field) of the last
        source update, or None when the noise is off."""
        nb = C.c_int32(0)
        self._check(self._lib.agis_get_attnoise(self.ctx, None, C.byref(nb)))
        if nb.value == 0:
            return None
        out = np.empty((3, nb.value), dtype=np.float64)
        self._check(self._lib.agis_get_attnoise(self.ctx, out.ctypes.data, C.byref(nb)))
        return out

    # source partitions: local sums, exchange, solve from the summed parts
    def exchange_size(self, which):
        n = C.c_int64(0)
        self._check(self._lib.agis_exchange_size(self.ctx, int(which), C.byref(n)))
        return n.value

    def accumulate(self, which):
        self._check(self._lib.agis_accumulate(self.ctx, int(which)))

    def get_exchange(self, which, out=None):
        """The context's partial sums into out (NumPy array or torch tensor, host or device)."""
        if out is None:
            out = np.empty(self.exchange_size(which), dtype=np.float64)
        self._check(self._lib.agis_get_exchange(self.ctx, int(which), _ptr(out)))
        return out

    def set_exchange(self, which, buf):
        self._check(self._lib.agis_set_exchange(self.ctx, int(which), _ptr(buf)))

    def solve_exchange(self, which):
        st = BlockStats()
        eo = np.zeros(6)
        self._check(self._lib.agis_solve_exchange(self.ctx, int(which), C.byref(st), eo.ctypes.data))
        d = st.as_dict()
        if which == X_FRAME:
            d["frame"] = eo
        return d


def _mlp_call(name, *args):
    lib = load()
    rc = getattr(lib, name)(*args)
    if rc != AGIS_OK:
        raise AgisError(rc, lib.agis_last_error(None).decode())


def _stream(stream):
    return C.c_void_p(stream) if stream is not None else None


def mlp_pack(params, packed, stream=None):
    """FP32 parameters (device) -> packed BF16 weights (device, MLP_PACKED_BYTES)."""
    _mlp_call("agis_mlp_pack", _ptr(params), _ptr(packed), _stream(stream))


def mlp_forward(packed, X, Y, stream=None):
    _mlp_call("agis_mlp_forward", _ptr(packed), _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream))


def mlp_loss_grad(params, X, T, grad, loss, idx=None, stream=None):
    n = int(idx.shape[0]) if idx is not None else int(X.shape[0])
    _mlp_call("agis_mlp_loss_grad", _ptr(params), _ptr(X), _ptr(T), _ptr(idx), n, _ptr(grad), _ptr(loss),
              _stream(stream))


def mlp_adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _mlp_call("agis_mlp_adam", _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr), float(beta1),
              float(beta2), float(eps), _stream(stream))


def proposal_targets(src_k, src_ref, sigma, T, stream=None):
    _mlp_call("agis_proposal_targets", _ptr(src_k), _ptr(src_ref), _ptr(sigma), int(src_k.shape[0]), _ptr(T),
              _stream(stream))


def _tune_dict(arr):
    return {KNOBS[e.knob]: dict(a=e.a, b=e.b, n_tried=e.n_tried, best_ms=e.best_ms, default_ms=e.default_ms)
            for e in arr}


def asi_estimate(d_prev, d_cur, stride, lambda_max, scratch, est, stream=None):
    """ASI estimate [median, lambda, factor, count] into est (4 FP64, device) from two
    n_src x 5 FP64 device updates; scratch: ceil(n_src / stride) x 8 bytes on the device."""
    _mlp_call("agis_asi_estimate", _ptr(d_prev), _ptr(d_cur), int(d_cur.shape[0]), int(stride), float(lambda_max),
              _ptr(scratch), _ptr(est), _stream(stream))


def obs_from_dataset(ds, device=None):
    """Observation arrays of a synth.Dataset, on the host or copied to a torch device (the gates
    with the full calibration model only)."""
    arrs = dict(t_ns=ds.t_ns, src=ds.src, ccd=ds.ccd, fov=ds.fov, kind=ds.kind, sigma=ds.sigma, mu=ds.mu)
    if ds.geometry.get("cal_generic"):
        arrs["gate"] = ds.gate
    if device is None:
        return {k: np.ascontiguousarray(v) for k, v in arrs.items()}
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in arrs.items()}


def calibration_config(geometry: dict) -> dict:
    """The agis_config fields of a dataset's calibration model."""
    if not geometry.get("cal_generic"):
        return dict(cal_model=0)
    return dict(cal_model=1, n_gate=int(geometry["n_gate"]), cal_j_per_k=int(geometry["cal_j_per_k"]),
                cal_col_bin=int(geometry["cal_col_bin"]))


def from_dataset(ds, cfg=None, device=None, with_ref=True, stream=None, **cfg_over):
    """Create a context from a synth.Dataset (starting values, truth as frame reference)."""
    if cfg is None:
        cfg = default_config(**{**calibration_config(ds.geometry), **cfg_over})
    ref = np.ascontiguousarray(ds.src_true[:, [0, 1, 3, 4]]) if with_ref else None
    return Agis(ds.geometry, cfg, obs_from_dataset(ds, device), np.ascontiguousarray(ds.src0),
                np.ascontiguousarray(ds.att0), np.ascontiguousarray(ds.cal0), src_ref=ref, stream=stream)


def source_update_static(geometry: dict, cfg: Config, obs: dict, src, att, cal, R_out=None, W_out=None,
                         stats_out=None, max_obs_per_source=STATIC_MAX_OBS, stream=None):
    """agis_source_update_static on device arrays (torch CUDA tensors); src is updated in place."""
    lib = load()
    o = Obs(*(_ptr(obs.get(k)) for k in ("t_ns", "src", "ccd", "fov", "kind", "sigma", "mu", "gate")))
    G = geometry_from_dict(geometry)
    s = C.c_void_p(stream) if stream is not None else None
    rc = lib.agis_source_update_static(C.byref(G), C.byref(cfg), C.byref(o), int(obs["t_ns"].shape[0]), _ptr(src),
                                       int(src.shape[0]), _ptr(att), _ptr(cal), _ptr(R_out), _ptr(W_out),
                                       _ptr(stats_out), int(max_obs_per_source), s)
    if rc != AGIS_OK:
        raise AgisError(rc, lib.agis_last_error(None).decode())
