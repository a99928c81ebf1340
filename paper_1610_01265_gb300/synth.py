"""Seeded synthetic coronal inputs on a logically rectangular spherical grid.

This module only *constructs inputs*: grid faces and the fields that the
frozen-coefficient operators take (temperature, magnetic direction, density,
viscosity, velocity).  It holds none of the method's arithmetic (no volumes,
areas, coefficients, stencils or integrators), so the CPU oracle and the CUDA
path can both consume its arrays without sharing any of the computation.

Layout of every scalar field: numpy float64 array of shape (nph, nth, nr),
C-order, so that r is the fastest index (the order of the paper's Fortran code,
Sec. 4.2).  Vector fields have shape (3, nph, nth, nr).

Field recipe (the stand-in for the paper's MAS coronal relaxation state,
Sec. 5 and Table 1, whose ADAPT map and restart files are not available):

* r faces geometric on [1, 2.5] R_sun with max/min spacing ratio 4, smallest
  spacing at r = 1; theta faces j*pi/nth; phi faces k*2*pi/nph (periodic).
* smooth seeded noise  xi(x) = sum_{q=1}^{12} a_q cos(k_q . x + p_q),  x the
  Cartesian position in R_sun, k_q integer components in [-3, 3],
  a_q ~ N(0,1), p_q ~ U[0, 2 pi), normalised to max|xi| = 1 on the grid.
* T = 1e6 K (1 + 0.5 tanh((r - 1.05)/0.02)) (1 + 0.05 xi_T)
* n = 1e8 r^-6 cm^-3
* B = dipole (2 cos(t), sin(t), 0)/r^3 plus a seeded quadrupole
  -grad(x^T Q x / |x|^5) scaled to 10% of the dipole's RMS on the r = 1 shell;
  bhat = B/|B| (bhat = rhat where |B| < 1e-12 max|B|).
* heating (a time sequence of backward-Euler steps): a source q(x, n) in K/s added
  explicitly before each implicit step n, q = q0 h(x) (1 + 0.25 sin(2 pi n / 50 + psi))
  with h = exp(-(r - 1)/0.3) (1 + 0.5 xi_h), psi ~ U[0, 2 pi); q0 is set by the caller.
* viscosity case: rho = m_p 1e8 r^-4, nu = 6.7e15 (1 + 0.1 xi_nu) cm^2/s, and a
  divergence-free v = curl(xi_1, xi_2, xi_3) in Cartesian components scaled to
  max|v| = 3e7 cm/s.
"""
from __future__ import annotations

import numpy as np

R_SUN_CM = 6.96e10
M_PROTON_G = 1.67262192e-24
NOISE_TERMS = 12


def r_faces(nr: int, r0: float = 1.0, r1: float = 2.5, ratio: float = 4.0) -> np.ndarray:
    """nr+1 radial faces (R_sun) with geometric spacing dr_i = dr_0 q^i, q = ratio^(1/(nr-1))."""
    if nr < 1:
        raise ValueError("nr must be >= 1")
    if nr == 1 or ratio == 1.0:
        return np.linspace(r0, r1, nr + 1)
    q = ratio ** (1.0 / (nr - 1))
    widths = q ** np.arange(nr)
    widths *= (r1 - r0) / widths.sum()
    rf = np.empty(nr + 1)
    rf[0] = r0
    rf[1:] = r0 + np.cumsum(widths)
    rf[-1] = r1
    return rf


def sample_points(nr: int, nth: int, nph: int, rf: np.ndarray):
    """Cell-centre sample coordinates (r, theta, phi) broadcast to (nph, nth, nr)."""
    rc = 0.5 * (rf[:-1] + rf[1:])
    tc = (np.arange(nth) + 0.5) * (np.pi / nth)
    pc = (np.arange(nph) + 0.5) * (2.0 * np.pi / nph)
    return (rc[None, None, :], tc[None, :, None], pc[:, None, None])


def _cartesian(r, t, p):
    st = np.sin(t)
    return r * st * np.cos(p), r * st * np.sin(p), r * np.cos(t) + 0.0 * p


def _noise_params(rng: np.random.Generator):
    k = rng.integers(-3, 4, size=(NOISE_TERMS, 3)).astype(np.float64)
    a = rng.standard_normal(NOISE_TERMS)
    ph = rng.uniform(0.0, 2.0 * np.pi, NOISE_TERMS)
    return k, a, ph


def _noise_eval(params, x, y, z, deriv: int | None = None):
    """xi (deriv=None) or d xi / d x_deriv at Cartesian points."""
    k, a, ph = params
    out = np.zeros(np.broadcast(x, y, z).shape)
    for q in range(NOISE_TERMS):
        arg = k[q, 0] * x + k[q, 1] * y + k[q, 2] * z + ph[q]
        if deriv is None:
            out += a[q] * np.cos(arg)
        else:
            out -= a[q] * k[q, deriv] * np.sin(arg)
    return out


def smooth_noise(rng: np.random.Generator, x, y, z) -> np.ndarray:
    """One seeded smooth noise field, normalised to max|xi| = 1 on the given points."""
    xi = _noise_eval(_noise_params(rng), x, y, z)
    m = np.max(np.abs(xi))
    return xi / m if m > 0 else xi


def _to_spherical(vx, vy, vz, t, p):
    st, ct, sp, cp = np.sin(t), np.cos(t), np.sin(p), np.cos(p)
    vr = vx * st * cp + vy * st * sp + vz * ct
    vt = vx * ct * cp + vy * ct * sp - vz * st
    vp = -vx * sp + vy * cp
    return vr, vt, vp


def _quadrupole_cart(Q, x, y, z):
    """-grad(x^T Q x / |x|^5) in Cartesian components."""
    r2 = x * x + y * y + z * z
    r = np.sqrt(r2)
    qx = Q[0, 0] * x + Q[0, 1] * y + Q[0, 2] * z
    qy = Q[1, 0] * x + Q[1, 1] * y + Q[1, 2] * z
    qz = Q[2, 0] * x + Q[2, 1] * y + Q[2, 2] * z
    xqx = x * qx + y * qy + z * qz
    r5 = r2 * r2 * r
    r7 = r5 * r2
    return (-2.0 * qx / r5 + 5.0 * xqx * x / r7,
            -2.0 * qy / r5 + 5.0 * xqx * y / r7,
            -2.0 * qz / r5 + 5.0 * xqx * z / r7)


def magnetic_direction(rng: np.random.Generator, nth: int, nph: int, r, t, p,
                       quad_fraction: float = 0.10) -> np.ndarray:
    """bhat (3, ...) in local (r, theta, phi) components: dipole + seeded quadrupole."""
    m = rng.standard_normal((3, 3))
    Q = 0.5 * (m + m.T)
    Q -= np.trace(Q) / 3.0 * np.eye(3)
    # scale on the r = 1 shell, area weights sin(theta) on the grid's own angles
    ts = (np.arange(nth) + 0.5) * (np.pi / nth)
    ps = (np.arange(nph) + 0.5) * (2.0 * np.pi / nph)
    T1, P1 = np.meshgrid(ts, ps, indexing="ij")
    w = np.sin(T1)
    xs, ys, zs = _cartesian(1.0, T1, P1)
    bqx, bqy, bqz = _quadrupole_cart(Q, xs, ys, zs)
    rms_q = np.sqrt(np.sum(w * (bqx**2 + bqy**2 + bqz**2)) / np.sum(w))
    rms_d = np.sqrt(np.sum(w * (4.0 * np.cos(T1) ** 2 + np.sin(T1) ** 2)) / np.sum(w))
    Q *= quad_fraction * rms_d / rms_q

    x, y, z = _cartesian(r, t, p)
    bqx, bqy, bqz = _quadrupole_cart(Q, x, y, z)
    bqr, bqt, bqp = _to_spherical(bqx, bqy, bqz, t, p)
    r3 = r**3
    br = 2.0 * np.cos(t) / r3 + bqr
    bt = np.sin(t) / r3 + bqt
    bp = bqp + 0.0 * br
    br, bt, bp = np.broadcast_arrays(br, bt, bp)
    mag = np.sqrt(br * br + bt * bt + bp * bp)
    tiny = mag < 1e-12 * np.max(mag)
    safe = np.where(tiny, 1.0, mag)
    out = np.stack([np.where(tiny, 1.0, br / safe),
                    np.where(tiny, 0.0, bt / safe),
                    np.where(tiny, 0.0, bp / safe)])
    return np.ascontiguousarray(out)


def conduction_case(nr: int, nth: int, nph: int, seed: int = 1) -> dict:
    """Seeded anisotropic-conduction inputs: rf, T (K), bhat, n (cm^-3)."""
    rng = np.random.default_rng(seed)
    rf = r_faces(nr)
    r, t, p = sample_points(nr, nth, nph, rf)
    x, y, z = _cartesian(r, t, p)
    xi_T = smooth_noise(rng, x, y, z)
    T = 1e6 * (1.0 + 0.5 * np.tanh((r - 1.05) / 0.02)) * (1.0 + 0.05 * xi_T)
    bhat = magnetic_direction(rng, nth, nph, r, t, p)
    n = np.broadcast_to(1e8 * r**-6, (nph, nth, nr))
    return {
        "shape": (nph, nth, nr),
        "rf": rf,
        "T": np.ascontiguousarray(T, dtype=np.float64),
        "bhat": bhat,
        "n": np.ascontiguousarray(n, dtype=np.float64),
        "kappa0": 9e-7,
    }


def viscosity_case(nr: int, nth: int, nph: int, seed: int = 1) -> dict:
    """Seeded viscosity inputs: rf, rho (g cm^-3), nu (cm^2/s), v (3, ...) Cartesian cm/s."""
    rng = np.random.default_rng(seed + 1000)
    rf = r_faces(nr)
    r, t, p = sample_points(nr, nth, nph, rf)
    x, y, z = _cartesian(r, t, p)
    xi_nu = smooth_noise(rng, x, y, z)
    nu = 6.7e15 * (1.0 + 0.1 * xi_nu)
    A = [_noise_params(rng) for _ in range(3)]
    d = lambda c, axis: _noise_eval(A[c], x, y, z, deriv=axis)  # noqa: E731
    vx = d(2, 1) - d(1, 2)
    vy = d(0, 2) - d(2, 0)
    vz = d(1, 0) - d(0, 1)
    vmax = np.max(np.sqrt(vx * vx + vy * vy + vz * vz))
    v = np.stack(np.broadcast_arrays(vx, vy, vz)) * (3e7 / vmax)
    rho = np.broadcast_to(M_PROTON_G * 1e8 * r**-4, (nph, nth, nr))
    return {
        "shape": (nph, nth, nr),
        "rf": rf,
        "rho": np.ascontiguousarray(rho, dtype=np.float64),
        "nu": np.array(np.broadcast_to(nu, (nph, nth, nr)), dtype=np.float64),
        "v": np.ascontiguousarray(v, dtype=np.float64),
    }


def heating_case(nr: int, nth: int, nph: int, seed: int = 1) -> dict:
    """Seeded heating pattern h (>= 0.5 exp(-(r-1)/0.3)) and phase psi of its modulation."""
    rng = np.random.default_rng(seed + 2000)
    rf = r_faces(nr)
    r, t, p = sample_points(nr, nth, nph, rf)
    x, y, z = _cartesian(r, t, p)
    xi = smooth_noise(rng, x, y, z)
    h = np.exp(-(r - 1.0) / 0.3) * (1.0 + 0.5 * xi)
    return {"h": np.ascontiguousarray(np.broadcast_to(h, (nph, nth, nr)), dtype=np.float64),
            "psi": float(rng.uniform(0.0, 2.0 * np.pi))}


def heating_modulation(step: int, psi: float) -> float:
    """Time factor of the heating source at step n."""
    return 1.0 + 0.25 * np.sin(2.0 * np.pi * step / 50.0 + psi)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform seeded test vector (used for operator parity and symmetry checks)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)
