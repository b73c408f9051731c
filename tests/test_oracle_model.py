"""Pins for the observation model and its partial derivatives (Sects. 3.2-3.6, 5.1.3, 5.2.3)."""
import numpy as np
import pytest

import synth
from oracle import model as M
from oracle import quat as Q


@pytest.fixture(scope="module")
def ds():
    return synth.simulate(synth.config("small1yr", n_src=400, noise_free=False))


def test_residuals_at_truth_equal_injected_noise(ds):
    # the simulator solves the observation times on its own (matrix-based) model; at the true
    # parameters the oracle's residuals must equal the noise it injected
    P = M.problem_from_dataset(ds)
    ev = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, partials=False)
    assert np.max(np.abs(ev["R"] - ds.noise)) < 2e-15


def test_normal_triad_and_special_cases():
    rng = np.random.default_rng(0)
    a, d = rng.uniform(0, 2 * np.pi, 100), rng.uniform(-1.5, 1.5, 100)
    p, q, r = M.normal_triad(a, d)
    for x, y in ((p, q), (q, r), (p, r)):
        assert np.allclose(np.sum(x * y, axis=1), 0, atol=1e-15)
    assert np.allclose(np.cross(r, p), q, atol=1e-15)       # q = r x p
    assert np.allclose(p[:, 2], 0)                          # p = <Z x r>


def test_coordinate_direction_at_epoch_without_parallax(ds):
    P = M.problem_from_dataset(ds)
    s5 = np.array([[1.0, 0.3, 0.0, 1e-7, -2e-7]])
    # at t_B = t_ep the proper-motion term vanishes; with parallax 0 u_bar = r exactly
    t = np.array([P.t_ep_ns])
    u, ubar, p, q, r, b, vc, tau = M.proper_direction(P, s5, t)
    ubar_ref = M.unit(r + tau[:, None] * (p * 1e-7 - q * 2e-7))
    assert np.allclose(ubar, ubar_ref, atol=1e-16)
    assert abs(tau[0]) < 600 / M.YEAR_S                      # only the Roemer delay remains


def test_source_partials_against_finite_differences(ds):
    P = M.problem_from_dataset(ds)
    idx = np.arange(0, P.n_obs, 53)
    ev = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, idx=idx)
    h = 1e-6
    for k in range(5):
        s1, s2 = ds.src_true.copy(), ds.src_true.copy()
        if k == 0:
            s1[:, 0] += h / np.cos(s1[:, 1])
            s2[:, 0] -= h / np.cos(s2[:, 1])
        else:
            s1[:, k] += h
            s2[:, k] -= h
        R1 = M.evaluate(P, s1, ds.att_true, ds.cal_true, idx=idx, partials=False)["R"]
        R2 = M.evaluate(P, s2, ds.att_true, ds.cal_true, idx=idx, partials=False)["R"]
        fd = -(R1 - R2) / (2 * h)
        # Eq. duds is accurate to better than 1e-6 (relative)
        assert np.max(np.abs(fd - ev["A"][:, k])) < 1e-6 * np.max(np.abs(ev["A"][:, k]))


def test_attitude_partials_against_finite_differences(ds):
    P = M.problem_from_dataset(ds)
    idx = np.arange(7, P.n_obs, 997)[:30]
    ev = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, idx=idx)
    G = M.attitude_design(ev)
    h = 1e-6
    for o in range(idx.size):
        l = ev["l"][o]
        for j in range(4):
            for c in range(4):
                a1, a2 = ds.att_true.copy(), ds.att_true.copy()
                a1[l - 3 + j, c] += h
                a2[l - 3 + j, c] -= h
                R1 = M.evaluate(P, ds.src_true, a1, ds.cal_true, idx=idx[o:o + 1], partials=False)["R"][0]
                R2 = M.evaluate(P, ds.src_true, a2, ds.cal_true, idx=idx[o:o + 1], partials=False)["R"][0]
                assert abs((R1 - R2) / (2 * h) - G[o, j, c]) < 1e-8


def test_attitude_partial_orthogonal_to_q(ds):
    # dR/dq is orthogonal to q, so the 1/||s|| factor is the exact normalisation derivative
    P = M.problem_from_dataset(ds)
    ev = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, idx=np.arange(0, P.n_obs, 11))
    dots = np.sum(ev["gq"] * ev["q"], axis=1)
    assert np.max(np.abs(dots)) < 1e-14


def test_field_angle_zero_on_the_viewing_direction(ds):
    P = M.problem_from_dataset(ds)
    q = Q.qunit(ds.att_true[100])
    for f in (1.0, -1.0):
        phi = f * P.gamma_c / 2
        us = np.array([np.cos(phi), np.sin(phi), 0.0])       # viewing direction in the SRS
        uc = Q.vector_rotate(q, us)                           # ICRS components
        ph, ze = M.field_angles(Q.frame_rotate(q, uc))
        assert abs(ph - phi) < 1e-15 and abs(ze) < 1e-15


def test_calibration_index_convention(ds):
    P = M.problem_from_dataset(ds)
    k = M.cal_index(P, ds.t_ns, ds.fov, ds.ccd, ds.kind)
    assert k.min() >= 0 and k.max() < P.n_cal
    al = ds.kind == 0
    assert np.all(k[al] < P.n_cal_days * 124) and np.all(k[~al] >= P.n_cal_days * 124)
