"""The simple iteration with the S[ACG] preconditioner (Sects. 4.5-4.6) and the frame
rotator applied after each iteration (Sect. 6.1.6), FP64."""
from dataclasses import dataclass

import numpy as np

from . import attnoise as AN
from . import blocks as B
from . import model as M


@dataclass
class State:
    src: np.ndarray   # [n_src, 5]
    att: np.ndarray   # [n_coef, 4]
    cal: np.ndarray   # [n_cal]
    eps2_a: np.ndarray = None   # excess attitude noise [3, n_buckets] (Sect. 5.2.5), or None

    def copy(self):
        return State(self.src.copy(), self.att.copy(), self.cal.copy(),
                     None if self.eps2_a is None else self.eps2_a.copy())


@dataclass
class IterStats:
    chi2: float            # sum_l W_l R_l^2 after the source update
    Q: float               # sum_i Q_i
    nu: int                # sum_i nu_i
    n_out: int
    rank_def_s: int
    rank_def_a: int
    rank_def_c: int
    frame: np.ndarray      # (eps, omega) applied, 6 values
    d_rms: np.ndarray      # RMS of the 5 source updates (rad, rad/yr)


def iterate_once(P, state, st, ref=None, after_s=None):
    """One AGIS iteration in the order of Sect. 4.6: s^(k+1) from a^(k), c^(k); then a^(k+1)
    and c^(k+1) both from s^(k+1) with the old a^(k), c^(k); then the frame rotator.
    st.block_order selects the variants of Sect. 4.6 (see blocks.Settings).
    after_s(src1, sres, ev) -> (src1, R), if given, changes the sources after the S block and
    returns the residuals the A and C blocks read (the accelerated iteration, Sect. 4.7)."""
    an = st.att_noise_bucket_ns > 0
    if an:
        # excess attitude noise (Sect. 5.2.5): the source update with sigma~^2 = sigma^2 +
        # eps_a^2 of the previous estimate (Eq. W), then eps_a^2 from its residuals (Eq. e09)
        sig2 = P.sigma.astype(np.float64) ** 2
        comp = AN.component(P.kind, P.fov)
        bucket = AN.bucket_of(P.t_ns, P.knot0_ns, st.att_noise_bucket_ns)
        n_b = int(bucket.max()) + 1
        eps2_a = state.eps2_a if state.eps2_a is not None else np.zeros((AN.N_COMP, n_b))
        src1, sres, ev = B.source_update(P, state.src, state.att, state.cal, st,
                                         sig2=AN.adjusted_variance(sig2, eps2_a, comp, bucket))
        eps2_i_obs = sres.eps2[P.src]
        eps2_a = AN.estimate(sres.R, sig2, eps2_i_obs, comp, bucket, n_b)
        W_att = AN.attitude_weights(sres.R, sig2, eps2_i_obs, eps2_a, comp, bucket, B._wfun(st))
    else:
        src1, sres, ev = B.source_update(P, state.src, state.att, state.cal, st)
    R = sres.R
    if after_s is not None:
        src1, R = after_s(src1, sres, ev)
    if st.block_order == "[SAC]":
        R = ev["R"]                     # Jacobi: the residuals at the previous iterate
    att1, rda = state.att.copy(), 0
    cal1, rdc = state.cal.copy(), 0
    if "A" in st.block_mask:
        att1, rda = B.attitude_update(P, state.att, ev, R, W_att if an else sres.W, st)
    Rc = R
    if st.block_order == "SAC":
        # Gauss-Seidel: C sees the attitude update through the linearised residuals,
        # R + (dR/da) (a^(k+1) - a^(k)) (the N_ca block of Eq. precond)
        Ga = M.attitude_design(ev).reshape(P.n_obs, 16)
        da = (att1 - state.att).reshape(-1)
        cols = 4 * (ev["l"][:, None] - 3) + np.arange(16)
        Rc = R + np.sum(Ga * da[cols], axis=1)
    if "C" in st.block_mask:
        cal1, rdc = B.calibration_update(P, state.cal, ev, Rc, sres.W)
    frame = np.zeros(6)
    if st.frame_each_iter and ref is not None:
        eps, om = B.frame_fit(P, src1, ref)
        src1 = B.frame_apply_sources(P, src1, eps, om)
        att1 = B.frame_apply_attitude(P, att1, eps, om)
        frame = np.concatenate([eps, om])
    stats = IterStats(
        chi2=float(np.sum(sres.W * sres.R ** 2)), Q=float(np.sum(sres.Qi)), nu=int(np.sum(sres.nu)),
        n_out=int(np.sum(sres.n_out)), rank_def_s=int(np.sum(sres.rank_def)), rank_def_a=int(rda),
        rank_def_c=int(rdc), frame=frame, d_rms=np.sqrt(np.mean(sres.d ** 2, axis=0)))
    return State(src1, att1, cal1, eps2_a if an else state.eps2_a), stats, sres


def iterate(P, state, st, n_iter, ref=None, callback=None):
    hist = []
    for k in range(n_iter):
        state, stats, _ = iterate_once(P, state, st, ref)
        hist.append(stats)
        if callback is not None:
            callback(k, state, stats)
    return state, hist


def source_errors(src, truth):
    """Per-parameter errors of the sources (alpha* as a true arc)."""
    e = np.asarray(src) - np.asarray(truth)
    e[:, 0] = (np.mod(e[:, 0] + np.pi, 2 * np.pi) - np.pi) * np.cos(np.asarray(truth)[:, 1])
    return e
