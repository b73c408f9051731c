"""Pins for the quaternion algebra (App. A) against closed forms and matrix algebra."""
import numpy as np

from oracle import quat as Q


def _rq(rng, n=50):
    return rng.normal(size=(n, 4))


def test_product_matches_vector_form():
    # Eq. quatmultvec: ab = {a x b + a b_w + b a_w, a_w b_w - a.b}
    rng = np.random.default_rng(1)
    a, b = _rq(rng), _rq(rng)
    ref_v = np.cross(a[:, :3], b[:, :3]) + a[:, :3] * b[:, 3:] + b[:, :3] * a[:, 3:]
    ref_w = a[:, 3] * b[:, 3] - np.sum(a[:, :3] * b[:, :3], axis=1)
    ab = Q.qmul(a, b)
    assert np.allclose(ab[:, :3], ref_v, atol=1e-14)
    assert np.allclose(ab[:, 3], ref_w, atol=1e-14)


def test_associative_and_norm():
    rng = np.random.default_rng(2)
    a, b, c = _rq(rng), _rq(rng), _rq(rng)
    assert np.allclose(Q.qmul(Q.qmul(a, b), c), Q.qmul(a, Q.qmul(b, c)), atol=1e-13)
    aa = Q.qmul(a, Q.qconj(a))
    assert np.allclose(aa[:, 3], np.sum(a * a, axis=1), atol=1e-13)
    assert np.allclose(aa[:, :3], 0, atol=1e-13)
    # (ab)* = b* a*, Eq. quatcom
    assert np.allclose(Q.qconj(Q.qmul(a, b)), Q.qmul(Q.qconj(b), Q.qconj(a)), atol=1e-13)


def test_frame_rotation_equals_attitude_matrix():
    # {S'v,0} = q^-1 {C'v,0} q equals A C'v with A from Eq. quat2mat
    rng = np.random.default_rng(3)
    q = Q.qunit(_rq(rng))
    v = rng.normal(size=(50, 3))
    A = Q.quat2mat(q)
    assert np.allclose(Q.frame_rotate(q, v), np.einsum("nij,nj->ni", A, v), atol=1e-14)
    # the matrix is proper orthonormal
    assert np.allclose(np.einsum("nij,nkj->nik", A, A), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(A), 1.0, atol=1e-14)


def test_rotation_about_z_closed_form():
    # rotation of the frame by theta about Z: x axis -> (cos, sin, 0) in the old frame
    th = 0.7
    q = Q.Q(np.array([0, 0, th]))
    A = Q.quat2mat(q)
    assert np.allclose(A[0], [np.cos(th), np.sin(th), 0], atol=1e-15)
    # a fixed vector appears rotated by -theta in the new frame
    v = np.array([1.0, 0, 0])
    assert np.allclose(Q.frame_rotate(q, v), [np.cos(th), -np.sin(th), 0], atol=1e-15)


def test_klumpp_round_trip():
    rng = np.random.default_rng(4)
    for q in Q.qunit(_rq(rng, 200)):
        q2 = Q.mat2quat(Q.quat2mat(q))
        s = np.sign(q[3]) if q[3] != 0 else 1.0
        assert np.allclose(q2, s * q, atol=1e-13)
        assert q2[3] >= 0


def test_successive_frame_rotations_compose_left_to_right():
    # Eq. quatframerot1: frame rotations q1 then q2 equal one rotation by q1 q2
    rng = np.random.default_rng(5)
    q1, q2 = Q.qunit(_rq(rng)), Q.qunit(_rq(rng))
    v = rng.normal(size=(50, 3))
    assert np.allclose(Q.frame_rotate(q2, Q.frame_rotate(q1, v)), Q.frame_rotate(Q.qmul(q1, q2), v), atol=1e-13)


def test_diffrot_small_angles():
    rng = np.random.default_rng(6)
    q0 = Q.qunit(_rq(rng))
    phi = rng.normal(size=(50, 3)) * 1e-6
    q1 = Q.qmul(q0, Q.Q(phi))
    assert np.allclose(Q.diffrot(q0, q1), phi, atol=1e-15, rtol=1e-9)
    # sign ambiguity handled by d_w
    assert np.allclose(Q.diffrot(q0, -q1), phi, atol=1e-15, rtol=1e-9)
