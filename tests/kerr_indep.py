"""Independent Kerr-geometry helpers for pinning the oracle.

Nothing here is taken from the paper's Appendix A: the Kerr metric is the
textbook Boyer-Lindquist form (Boyer & Lindquist 1967; e.g. Misner, Thorne &
Wheeler eq. 33.2), moved to Kerr-Schild coordinates with the coordinate
differentials of the paper's Eq. BL_KS_diff (dt_KS = dt_BL + 2r/Delta dr,
dphi_KS = dphi_BL + a/Delta dr), and inverted numerically with numpy.
Coordinates are ordered (t, r, theta, phi)."""
import math
import numpy as np


def g_bl(a, r, th):
    s, c = math.sin(th), math.cos(th)
    Sig = r * r + a * a * c * c
    Dl = r * r - 2 * r + a * a
    g = np.zeros((4, 4))
    g[0, 0] = -(1 - 2 * r / Sig)
    g[0, 3] = g[3, 0] = -2 * a * r * s * s / Sig
    g[1, 1] = Sig / Dl
    g[2, 2] = Sig
    g[3, 3] = (r * r + a * a + 2 * a * a * r * s * s / Sig) * s * s
    return g


def g_ks(a, r, th):
    """g_{mu nu} in Kerr-Schild coordinates: g_KS = J^T g_BL J with
    J = d x_BL / d x_KS (only the r column has off-diagonal entries)."""
    Dl = r * r - 2 * r + a * a
    J = np.eye(4)
    J[0, 1] = -2 * r / Dl
    J[3, 1] = -a / Dl
    return J.T @ g_bl(a, r, th) @ J


def ginv_ks(a, r, th):
    return np.linalg.inv(g_ks(a, r, th))


def three_plus_one(a, r, th):
    """alpha, beta^i, gamma_ij, gamma^ij from the 4-metric (standard 3+1
    identities: g^tt = -1/alpha^2, g^ti = beta^i/alpha^2)."""
    g = g_ks(a, r, th)
    gi = np.linalg.inv(g)
    alpha = 1.0 / math.sqrt(-gi[0, 0])
    beta = gi[0, 1:] * alpha * alpha
    gam = g[1:, 1:]
    return alpha, beta, gam, np.linalg.inv(gam)


def u_t(a, r, th, ui, eps=1.0):
    """Covariant u_t from g^{mu nu} u_mu u_nu = -eps, future-directed root."""
    gi = ginv_ks(a, r, th)
    uu = np.array([0.0, *ui])
    A = gi[0, 0]
    B = 2 * gi[0, 1:] @ np.asarray(ui)
    Cc = np.asarray(ui) @ gi[1:, 1:] @ np.asarray(ui) + eps
    disc = math.sqrt(B * B - 4 * A * Cc)
    r1, r2 = (-B + disc) / (2 * A), (-B - disc) / (2 * A)
    # future directed: u^t = g^{t mu} u_mu > 0
    for cand in (r1, r2):
        uu[0] = cand
        if gi[0] @ uu > 0:
            return cand
    raise ValueError("no future-directed root")


def energy(a, y, eps=1.0):
    """E = -u_t for state y = (r, theta, phi, u_r, u_theta, u_phi)."""
    return -u_t(a, y[0], y[1], y[3:6], eps)


def carter_Q(a, y, eps=1.0):
    """Carter constant Q = u_theta^2 + cos^2(theta) (a^2 (eps - E^2) + L^2 / sin^2(theta));
    u_theta, u_t, u_phi agree between BL and KS coordinates."""
    E = energy(a, y, eps)
    L = y[5]
    th = y[1]
    return y[4] ** 2 + math.cos(th) ** 2 * (a * a * (eps - E * E) + L * L / math.sin(th) ** 2)


def hamilton_rhs(a, y, eps=1.0, h=1e-3):
    """dx^i/dt and du_i/dt of a geodesic from Hamilton's equations with
    H = g^{mu nu} u_mu u_nu / 2 (u_t held at its conserved value):
    dx^i/dt = g^{i mu} u_mu / u^t,  du_i/dt = -(d_i g^{mu nu}) u_mu u_nu / (2 u^t);
    the metric derivative is a 4th-order central difference."""
    r, th = y[0], y[1]
    ut = u_t(a, r, th, y[3:6], eps)
    u = np.array([ut, y[3], y[4], y[5]])
    gi = ginv_ks(a, r, th)
    ut_up = gi[0] @ u
    dx = (gi[1:] @ u) / ut_up

    def dgi(k):
        def at(d):
            rr, tt = (r + d, th) if k == 0 else (r, th + d)
            return ginv_ks(a, rr, tt)
        return (-at(2 * h) + 8 * at(h) - 8 * at(-h) + at(-2 * h)) / (12 * h)

    du = np.array([-(u @ dgi(0) @ u) / (2 * ut_up), -(u @ dgi(1) @ u) / (2 * ut_up), 0.0])
    return np.concatenate([dx, du])


def load_table1(path):
    rows = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        name = f[0]
        th = eval(f[7], {"pi": math.pi})
        rows[name] = dict(a=float(f[1]), Bz=float(f[2]), u=(float(f[3]), float(f[4]), float(f[5])),
                          r=float(f[6]), th=th)
    return rows
