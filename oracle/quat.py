"""Quaternion algebra, App. A of the paper.  Quaternions are arrays [..., 4]
holding {x, y, z, w} (vector part first, Sect. A.1)."""
import numpy as np


def qmul(a, b):
    """Product ab, Eq. quatmult."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ax, ay, az, aw = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bx, by, bz, bw = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([
        ax * bw + ay * bz - az * by + aw * bx,
        -ax * bz + ay * bw + az * bx + aw * by,
        ax * by - ay * bx + az * bw + aw * bz,
        -ax * bx - ay * by - az * bz + aw * bw,
    ], axis=-1)


def qconj(a):
    """Conjugate, Eq. quatconj."""
    a = np.asarray(a, dtype=np.float64)
    return np.concatenate([-a[..., :3], a[..., 3:]], axis=-1)


def qnorm(a):
    """Norm, Eq. quatnorm."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(np.sum(a * a, axis=-1))


def qinv(a):
    """Inverse, Eq. quatinv."""
    return qconj(a) / (qnorm(a) ** 2)[..., None]


def qunit(a):
    """Normalisation <a>, Eq. vecquatnorm."""
    return np.asarray(a, dtype=np.float64) / qnorm(a)[..., None]


def vq(v):
    """The pure quaternion {v, 0}."""
    v = np.asarray(v, dtype=np.float64)
    return np.concatenate([v, np.zeros(v.shape[:-1] + (1,))], axis=-1)


def Q(phi):
    """Unit quaternion of the rotation by |phi| about phi, Eq. qrot."""
    phi = np.asarray(phi, dtype=np.float64)
    ang = np.sqrt(np.sum(phi * phi, axis=-1))
    out = np.zeros(phi.shape[:-1] + (4,))
    out[..., 3] = 1.0
    nz = ang > 0
    if np.any(nz):
        s = np.sin(0.5 * ang[nz]) / ang[nz]
        out[nz, :3] = phi[nz] * s[..., None]
        out[nz, 3] = np.cos(0.5 * ang[nz])
    return out


def frame_rotate(q, v):
    """Coordinates of v in the frame rotated by q: {S1'v,0} = q^-1 {S0'v,0} q, Eq. quatframerot."""
    return qmul(qmul(qinv(q), vq(v)), q)[..., :3]


def vector_rotate(q, v):
    """Vector rotation {S'r1,0} = q {S'r0,0} q^-1, Eq. quatvecrot."""
    return qmul(qmul(q, vq(v)), qinv(q))[..., :3]


def quat2mat(q):
    """Attitude matrix from a unit quaternion, Eq. quat2mat."""
    q = np.asarray(q, dtype=np.float64)
    x, y, z, w = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    m = np.empty(q.shape[:-1] + (3, 3))
    m[..., 0, 0] = 1 - 2 * (y * y + z * z)
    m[..., 0, 1] = 2 * (x * y + z * w)
    m[..., 0, 2] = 2 * (x * z - y * w)
    m[..., 1, 0] = 2 * (x * y - z * w)
    m[..., 1, 1] = 1 - 2 * (x * x + z * z)
    m[..., 1, 2] = 2 * (y * z + x * w)
    m[..., 2, 0] = 2 * (x * z + y * w)
    m[..., 2, 1] = 2 * (y * z - x * w)
    m[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return m


def mat2quat(A):
    """Unit quaternion (q_w >= 0) from an attitude matrix, Algorithm A.1 (Klumpp 1976)."""
    A = np.asarray(A, dtype=np.float64)
    s = A[0, 0] + A[1, 1] + A[2, 2]
    mag = [np.sqrt(max((1 - s) / 4 + A[i, i] / 2, 0.0)) for i in range(3)]
    qw = np.sqrt(max((1 + s) / 4, 0.0))
    if mag[0] >= max(mag[1], mag[2]):
        i, j, k = 0, 1, 2
    elif mag[1] >= max(mag[0], mag[2]):
        i, j, k = 1, 2, 0
    else:
        i, j, k = 2, 0, 1
    q = np.zeros(4)
    q[i] = mag[i] * np.sign(A[j, k] - A[k, j])
    q[j] = mag[j] * np.sign(q[i] * (A[i, j] + A[j, i]))
    q[k] = mag[k] * np.sign(q[i] * (A[i, k] + A[k, i]))
    q[3] = qw
    return q


def diffrot(q0, q1):
    """Small rotation angles (phi_x, phi_y, phi_z) from S0 to S1, Eqs. diffrot2-diffrot3."""
    d = qmul(qinv(q0), q1)
    return 2.0 * d[..., :3] * d[..., 3:4]
