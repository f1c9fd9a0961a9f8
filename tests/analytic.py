"""Closed forms used as pins (Sec. 4.1 analytic model of the standing wave,
Young-Laplace jump, plane Poiseuille flow).  Written from the equations; no
simulation code."""
import math


def wave_setting(L: int, omega: float = 1.8, re: float = 10.0):
    """Paper setting of the gravity wave (Sec. 4.1): tau = 1/omega, nu from
    Eq. nm-lbm-viscosity, omega0 from Re = a0 omega0 L / nu, g from the
    dispersion relation omega0^2 = g k tanh(k d)."""
    nu = (1.0 / 3.0) * (1.0 / omega - 0.5)
    k = 2.0 * math.pi / L
    d = L / 2.0
    a0 = 0.01 * L
    w0 = re * nu / (a0 * L)
    g = w0 * w0 / (k * math.tanh(k * d))
    return dict(nu=nu, k=k, d=d, a0=a0, omega0=w0, g=g)


def omega0(g: float, k: float, d: float) -> float:
    return math.sqrt(g * k * math.tanh(k * d))


def amplitude(t: float, a0: float, nu: float, k: float, w0: float) -> float:
    """a(0, t) - d = a0 exp(-2 nu k^2 t) cos(omega0 t)."""
    return a0 * math.exp(-2.0 * nu * k * k * t) * math.cos(w0 * t)


def log_decrement(nu: float, k: float, w0: float) -> float:
    """ln(a(t) / a(t + T)) with T = 2 pi / omega0."""
    return 2.0 * nu * k * k * (2.0 * math.pi / w0)


def poiseuille(y: float, H: float, g: float, nu: float) -> float:
    """Body-force driven channel between walls at 0 and H: u = g y (H - y) / (2 nu)."""
    return g * y * (H - y) / (2.0 * nu)
