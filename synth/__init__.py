"""Seeded synthetic Gaia-like data for the AGIS hot path.

This package is the input generator shared by the FP64 oracle (``oracle/``), the
GPU library (``paper_1112_4139_gb300``), the tests and ``bench.py``.  It holds a
simulation of the sky, the scanning instrument and its observations (the role
played by the Gaia System Simulator for the demonstration solution of
Lindegren et al. 2012, Sect. 7.2) and none of the solution method: no residual
weighting, partial derivatives, normal equations or solvers.

Recipe (readings of the paper where it is silent):
  * sources: alpha ~ U[0, 2pi), sin(delta) ~ U[-1, 1], parallax ~ Exp(mean 1 mas),
    mu_alpha*, mu_delta ~ N(0, 10 mas/yr); G ~ U(12, 18) for the
    magnitude-dependent workload with sigma_AL = 50 uas * 10^((G-12)/6) and
    sigma_AC = 5.65 sigma_AL; otherwise sigma_AL = 100 uas, sigma_AC = 500 uas.
  * scanning law: uniformly revolving, solar aspect 45 deg, spin 60 arcsec/s,
    5.8 precessions per year, basic angle 106.5 deg.
  * ephemeris: circular 1-AU orbit in the ecliptic, J2000 obliquity.
  * attitude: cubic B-spline (uniform knots, 4-fold end knots) obtained by a
    cubic quasi-interpolant of the scanning law followed by a smooth
    perturbation (8 sinusoids per axis, periods 4-48 knot intervals, 10 arcsec
    total RMS).  The spline itself is the truth.
  * focal plane: 7 AC rows x 9 AL strips without (row 3, strip 8) = 62 AF CCDs;
    9 AL observations per field transit (8 in row 3) and 1 AC observation on
    the first strip of the row.
  * calibration: per (field, CCD, day) AL offsets N(0, 0.5 mas) and per
    (field, row, day) AC offsets N(0, 5 mas), projected onto the constraints
    (zero mean over the 124 AL offsets of a day, over the 7 AC offsets of a
    field and day).
  * full geometric calibration (cal_generic): the terms of Eq. etazeta per CCD and gate in the
    layout of oracle/calgeneric.py (r = 0 AL terms N(0, 0.5 mas), r = 1, 2 terms N(0, 0.1 mas),
    small-scale AL terms N(0, 0.05 mas), r = 0 AC terms N(0, 5 mas) on the AF1 CCDs, made to
    satisfy Eqs. cc1-cc3); an observation of a source of magnitude G is gated when G plus a
    N(0, 0.15 mag) jitter is below 13 (gate 1 + floor((13 - G') / 0.5)); AL observations record
    the AC pixel coordinate of the image (mu from the nominal AC line at the true zeta).
  * observables: the crossing time of the calibrated observation line is solved
    on the true model, so that the residual at truth equals the injected noise
    (Gaussian, plus 1% of components offset by +-10 sigma); times are rounded
    to integer nanoseconds.  AC: the pixel coordinate mu is solved likewise.
  * starting values: sources truth + N(0, 50 mas) in alpha*, delta with zero
    parallax and proper motion; attitude truth with each coefficient rotated by
    an independent N(0, 50 mas) rotation per axis; calibration zero.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gaia_sim.c")
_LIB = os.path.join(_HERE, "libgaia_sim.so")
_lock = threading.Lock()
_lib = None

ARCSEC = np.pi / 648000.0
MAS = ARCSEC * 1e-3
UAS = ARCSEC * 1e-6
DAY_NS = 86_400 * 1_000_000_000
YEAR_S = 365.25 * 86400.0
YEAR_NS = int(round(YEAR_S * 1e9))
N_CCD = 62
N_ROW = 7


class _SimConfig(C.Structure):
    _fields_ = [
        ("n_src", C.c_int64), ("span_ns", C.c_int64), ("knot_dt_ns", C.c_int64), ("cal_dt_ns", C.c_int64),
        ("seed", C.c_uint64), ("sigma_al", C.c_double), ("sigma_ac", C.c_double),
        ("mag_dependent", C.c_int32), ("noise_free", C.c_int32),
        ("outlier_frac", C.c_double), ("outlier_nsigma", C.c_double), ("att_pert_rms", C.c_double),
        ("cal_al_rms", C.c_double), ("cal_ac_rms", C.c_double), ("start_src_err", C.c_double),
        ("start_att_err", C.c_double), ("min_transits", C.c_int32), ("max_transits", C.c_int32),
        ("dec_min", C.c_double), ("dec_max", C.c_double), ("ra_min", C.c_double), ("ra_max", C.c_double),
        ("parallax_mean", C.c_double), ("pm_sigma", C.c_double), ("n_threads", C.c_int32),
        ("cal_generic", C.c_int32), ("n_gate", C.c_int32), ("cal_j_per_k", C.c_int32), ("cal_col_bin", C.c_int32),
        ("gate_g0", C.c_double), ("gate_step", C.c_double), ("gate_fuzz", C.c_double),
        ("cal_l12_rms", C.c_double), ("cal_small_rms", C.c_double),
    ]


class _SimGeometry(C.Structure):
    _fields_ = [
        ("gamma_c", C.c_double), ("focal_length", C.c_double), ("p_ac", C.c_double), ("mu_c", C.c_double),
        ("eta0", C.c_double * N_CCD), ("x_fpa", C.c_double * N_CCD), ("x_centre", C.c_double * 2),
        ("ccd_row", C.c_int32 * N_CCD), ("ccd_strip", C.c_int32 * N_CCD),
        ("xi", C.c_double), ("spin_rate", C.c_double), ("prec_rate", C.c_double),
        ("spin0", C.c_double), ("prec0", C.c_double),
        ("orb_L0", C.c_double), ("obliquity", C.c_double), ("cos_obl", C.c_double), ("sin_obl", C.c_double),
        ("au_light_s", C.c_double), ("t_ep_ns", C.c_int64), ("t_fr_ns", C.c_int64),
        ("knot0_ns", C.c_int64), ("n_coef", C.c_int64), ("n_cal_days", C.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile the simulator with the host C compiler (OpenMP when available)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["cc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            cmd.remove("-fopenmp")
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("simulator build failed:\n" + r.stderr)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        lib.sim_create.restype = C.c_void_p
        lib.sim_create.argtypes = [C.POINTER(_SimConfig)]
        lib.sim_generate.restype = C.c_int64
        lib.sim_generate.argtypes = [C.c_void_p]
        for f in ("sim_n_src_out", "sim_n_coef", "sim_n_cal"):
            getattr(lib, f).restype = C.c_int64
            getattr(lib, f).argtypes = [C.c_void_p]
        lib.sim_get_geometry.argtypes = [C.c_void_p, C.POINTER(_SimGeometry)]
        P = C.c_void_p
        lib.sim_copy_obs.argtypes = [C.c_void_p] + [P] * 8
        lib.sim_copy_truth.argtypes = [C.c_void_p] + [P] * 5
        lib.sim_copy_gate.argtypes = [C.c_void_p, P]
        lib.sim_starting_values.argtypes = [C.c_void_p] + [P] * 3
        lib.sim_field_angles.argtypes = [C.c_void_p, P, C.c_int64, P, P]
        lib.sim_target_quat.argtypes = [C.c_void_p, C.c_double, P]
        lib.sim_destroy.argtypes = [C.c_void_p]
        lib.sim_sizeof_config.restype = C.c_int
        lib.sim_sizeof_geometry.restype = C.c_int
        assert lib.sim_sizeof_config() == C.sizeof(_SimConfig), "sim_config layout mismatch"
        assert lib.sim_sizeof_geometry() == C.sizeof(_SimGeometry), "sim_geometry layout mismatch"
        _lib = lib
    return _lib


@dataclasses.dataclass
class SimConfig:
    """Workload description (sizes and noise model)."""
    name: str = "custom"
    n_src: int = 1000
    span_days: float = 365.25
    knot_dt_s: int = 3600
    cal_dt_s: int = 86400
    seed: int = 1112
    sigma_al: float = 100 * UAS
    sigma_ac: float = 500 * UAS
    mag_dependent: bool = False
    noise_free: bool = False
    outlier_frac: float = 0.01
    outlier_nsigma: float = 10.0
    att_pert_rms: float = 10 * ARCSEC
    cal_al_rms: float = 0.5 * MAS
    cal_ac_rms: float = 5 * MAS
    start_src_err: float = 50 * MAS
    start_att_err: float = 50 * MAS
    min_transits: int = 0
    max_transits: int = 0
    dec_range: tuple = (-np.pi / 2, np.pi / 2)
    ra_range: tuple = (0.0, 2 * np.pi)
    parallax_mean: float = 1 * MAS
    pm_sigma: float = 10 * MAS
    n_threads: int = 0
    # the full geometric calibration of Eq. etazeta instead of per-day offsets
    cal_generic: bool = False
    n_gate: int = 1
    cal_j_per_k: int = 1
    cal_col_bin: int = 1
    gate_g0: float = 13.0
    gate_step: float = 0.5
    gate_fuzz: float = 0.15
    cal_l12_rms: float = 0.1 * MAS
    cal_small_rms: float = 0.05 * MAS

    def span_ns(self) -> int:
        # whole number of knot intervals
        k = int(round(self.span_days * 86400.0 / self.knot_dt_s))
        return k * self.knot_dt_s * 1_000_000_000


@dataclasses.dataclass
class Dataset:
    cfg: SimConfig
    geometry: dict
    # observations, sorted by source then time
    t_ns: np.ndarray
    src: np.ndarray
    ccd: np.ndarray
    fov: np.ndarray
    kind: np.ndarray
    sigma: np.ndarray
    mu: np.ndarray
    noise: np.ndarray   # residual at truth (injected noise + ns rounding), for tests only
    # truth
    src_true: np.ndarray
    src_mag: np.ndarray
    n_transits: np.ndarray
    att_true: np.ndarray
    cal_true: np.ndarray
    # starting values
    src0: np.ndarray
    att0: np.ndarray
    cal0: np.ndarray
    gate: np.ndarray = None   # per observation (0: not gated); all 0 unless cfg.cal_generic

    @property
    def n_obs(self) -> int:
        return int(self.t_ns.shape[0])

    @property
    def n_src(self) -> int:
        return int(self.src_true.shape[0])

    @property
    def n_coef(self) -> int:
        return int(self.att_true.shape[0])

    @property
    def n_cal(self) -> int:
        return int(self.cal_true.shape[0])

    def src_offsets(self) -> np.ndarray:
        """Start index of every source's observations (length n_src + 1)."""
        return np.searchsorted(self.src, np.arange(self.n_src + 1)).astype(np.int64)

    def subset_sources(self, idx) -> "Dataset":
        """Dataset restricted to the given sources (attitude and calibration kept whole)."""
        idx = np.asarray(idx, dtype=np.int64)
        remap = -np.ones(self.n_src, dtype=np.int64)
        remap[idx] = np.arange(idx.size)
        keep = remap[self.src] >= 0
        order = np.argsort(remap[self.src[keep]], kind="stable")

        def sel(a):
            return np.ascontiguousarray(a[keep][order])
        return dataclasses.replace(
            self, t_ns=sel(self.t_ns), src=sel(remap[self.src]).astype(np.int32), ccd=sel(self.ccd),
            fov=sel(self.fov), kind=sel(self.kind), sigma=sel(self.sigma), mu=sel(self.mu),
            noise=sel(self.noise), gate=sel(self.gate), src_true=self.src_true[idx].copy(),
            src_mag=self.src_mag[idx].copy(),
            n_transits=self.n_transits[idx].copy(), src0=self.src0[idx].copy())


def simulate(cfg: SimConfig) -> Dataset:
    lib = _load()
    c = _SimConfig()
    c.n_src = cfg.n_src
    c.span_ns = cfg.span_ns()
    c.knot_dt_ns = cfg.knot_dt_s * 1_000_000_000
    c.cal_dt_ns = cfg.cal_dt_s * 1_000_000_000
    c.seed = cfg.seed
    c.sigma_al, c.sigma_ac = cfg.sigma_al, cfg.sigma_ac
    c.mag_dependent = int(cfg.mag_dependent)
    c.noise_free = int(cfg.noise_free)
    c.outlier_frac, c.outlier_nsigma = cfg.outlier_frac, cfg.outlier_nsigma
    c.att_pert_rms = cfg.att_pert_rms
    c.cal_al_rms, c.cal_ac_rms = cfg.cal_al_rms, cfg.cal_ac_rms
    c.start_src_err, c.start_att_err = cfg.start_src_err, cfg.start_att_err
    c.min_transits, c.max_transits = cfg.min_transits, cfg.max_transits
    c.dec_min, c.dec_max = cfg.dec_range
    c.ra_min, c.ra_max = cfg.ra_range
    c.parallax_mean, c.pm_sigma = cfg.parallax_mean, cfg.pm_sigma
    c.n_threads = cfg.n_threads
    c.cal_generic = int(cfg.cal_generic)
    c.n_gate, c.cal_j_per_k, c.cal_col_bin = cfg.n_gate, cfg.cal_j_per_k, cfg.cal_col_bin
    c.gate_g0, c.gate_step, c.gate_fuzz = cfg.gate_g0, cfg.gate_step, cfg.gate_fuzz
    c.cal_l12_rms, c.cal_small_rms = cfg.cal_l12_rms, cfg.cal_small_rms
    h = lib.sim_create(C.byref(c))
    try:
        n_obs = lib.sim_generate(h)
        n_src = lib.sim_n_src_out(h)
        n_coef = lib.sim_n_coef(h)
        n_cal = lib.sim_n_cal(h)
        g = _SimGeometry()
        lib.sim_get_geometry(h, C.byref(g))
        t_ns = np.empty(n_obs, np.int64)
        src = np.empty(n_obs, np.int32)
        ccd = np.empty(n_obs, np.uint8)
        fov = np.empty(n_obs, np.uint8)
        kind = np.empty(n_obs, np.uint8)
        sigma = np.empty(n_obs, np.float32)
        mu = np.empty(n_obs, np.float64)
        noise = np.empty(n_obs, np.float64)
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
        lib.sim_copy_obs(h, ptr(t_ns), ptr(src), ptr(ccd), ptr(fov), ptr(kind), ptr(sigma), ptr(mu), ptr(noise))
        gate = np.empty(n_obs, np.uint8)
        lib.sim_copy_gate(h, ptr(gate))
        src_true = np.empty((n_src, 5))
        src_mag = np.empty(n_src)
        n_tr = np.empty(n_src, np.int32)
        att_true = np.empty((n_coef, 4))
        cal_true = np.empty(n_cal)
        lib.sim_copy_truth(h, ptr(src_true), ptr(src_mag), ptr(att_true), ptr(cal_true), ptr(n_tr))
        src0 = np.empty((n_src, 5))
        att0 = np.empty((n_coef, 4))
        cal0 = np.empty(n_cal)
        lib.sim_starting_values(h, ptr(src0), ptr(att0), ptr(cal0))
    finally:
        lib.sim_destroy(h)
    geometry = dict(
        gamma_c=g.gamma_c, focal_length=g.focal_length, p_ac=g.p_ac, mu_c=g.mu_c,
        eta0=np.array(g.eta0[:]), x_fpa=np.array(g.x_fpa[:]), x_centre=np.array(g.x_centre[:]),
        ccd_row=np.array(g.ccd_row[:]), ccd_strip=np.array(g.ccd_strip[:]),
        orb_L0=g.orb_L0, obliquity=g.obliquity, au_light_s=g.au_light_s, year_s=YEAR_S,
        t_ep_ns=g.t_ep_ns, t_fr_ns=g.t_fr_ns, knot0_ns=g.knot0_ns, knot_dt_ns=c.knot_dt_ns,
        n_coef=g.n_coef, cal_t0_ns=0, cal_dt_ns=c.cal_dt_ns, n_cal_days=g.n_cal_days,
        span_ns=c.span_ns, spin_rate=g.spin_rate,
    )
    if cfg.cal_generic:
        geometry.update(cal_generic=1, n_gate=cfg.n_gate, cal_j_per_k=cfg.cal_j_per_k, cal_col_bin=cfg.cal_col_bin,
                        n_col=1966)
    return Dataset(cfg=cfg, geometry=geometry, t_ns=t_ns, src=src, ccd=ccd, fov=fov, kind=kind, sigma=sigma,
                   mu=mu, noise=noise, src_true=src_true, src_mag=src_mag, n_transits=n_tr, att_true=att_true,
                   cal_true=cal_true, src0=src0, att0=att0, cal0=cal0, gate=gate)


def config(name: str, **over) -> SimConfig:
    """Named workloads.

    small1yr : 10,000 sources, 1 yr, 1-h knots (plain FP64 block iteration, small)
    scale5yr : 1,000,000 sources, 5 yr, 30-s knots (plain FP64 at scale; also the
               mixed-precision workload)
    uneven5yr: 3,000,000 sources, magnitude-dependent sigma, 40-250 transits
    tiny     : a few hundred sources in a declination band, 10 days (tests)
    """
    base = dict(
        small1yr=dict(n_src=10_000, span_days=365.25, knot_dt_s=3600, seed=1112 + 1),
        scale5yr=dict(n_src=1_000_000, span_days=5 * 365.25, knot_dt_s=30, seed=1112 + 2),
        uneven5yr=dict(n_src=3_000_000, span_days=5 * 365.25, knot_dt_s=30, seed=1112 + 4, mag_dependent=True,
                       min_transits=40, max_transits=250),
        tiny=dict(n_src=400, span_days=10, knot_dt_s=3600, seed=7),
    )[name]
    base.update(over)
    return SimConfig(name=name, **base)
