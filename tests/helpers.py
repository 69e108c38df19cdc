"""Shared test plumbing: build oracle lattices from the seeded workloads, and measure errors."""
import numpy as np

from oracle import OracleLattice, TimeFn


def oracle_time_fn(fn):
    return TimeFn(fn.kind, fn.amplitude, fn.period, fn.phase, fn.table)


def oracle_from_workload(w, threads=1, eps0=0.0, mu0=0.0, init=True):
    L = OracleLattice(w.model, w.shape, w.eps_r, w.mu_r, w.sigma, eps0=eps0, mu0=mu0, threads=threads)
    for s in w.sources:
        if s.kind == "current":
            L.add_current(s.cells, s.w, oracle_time_fn(s.fn))
        else:
            L.add_impose(s.cells, s.E0, s.B0, oracle_time_fn(s.fn))
    if init:
        E = np.zeros((3, w.n)) if w.E is None else w.E
        B = np.zeros((3, w.n)) if w.B is None else w.B
        L.init_fields(E, B)
    return L


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


def peak_interp(y):
    """Signed value at the largest |y| sample, refined by a parabola through its two neighbours."""
    i = int(np.argmax(np.abs(y)))
    if i == 0 or i == len(y) - 1:
        return float(y[i])
    ym, y0, yp = y[i - 1], y[i], y[i + 1]
    den = ym - 2 * y0 + yp
    if den == 0:
        return float(y0)
    off = 0.5 * (ym - yp) / den
    return float(y0 - 0.25 * (ym - yp) * off)


def fresnel_interface_errors(run, model, lz):
    """Section IV-A on a 1 x 1 x Lz lattice: Gaussian pulse (eq. Initialpulse) at z0 = Lz/2 - Lz/6
    with alpha = 0.05 Lz / sqrt(2), eps_r = 2.5 for z >= Lz/2. Returns the relative errors of the
    reflected and transmitted peak amplitudes against Fresnel, measured 0.3 Lz / C after the pulse
    reaches the interface. ``run(eps_r, E, B, steps)`` returns E_x after that many steps."""
    from paper_2309_08068_gb300 import workloads as wl
    c = wl.LIGHT_SPEED[model]
    z = np.arange(lz, dtype=np.float64)
    eps = np.where(z >= lz / 2, 2.5, 1.0)
    alpha = 0.05 * lz / np.sqrt(2.0)
    E, B = wl.gaussian_pulse_fields(model, z, lz / 2 - lz / 6, alpha, 1.0)
    ex = np.asarray(run(eps, E, B, int(round((lz / 6) / c + 0.3 * lz / c))), dtype=np.float64)
    r = np.sqrt(2.5)
    R, T = -(r - 1) / (r + 1), 2 / (r + 1)
    a_r = peak_interp(ex[: lz // 2 - int(2 * alpha)])
    a_t = peak_interp(ex[lz // 2 + int(alpha):])
    return abs(a_r - R) / abs(R), abs(a_t - T) / T


def f24_value(x, scale):
    """The value FP32 x keeps under 24-bit population storage with a power-of-two scale, written
    out from the encoding's definition: h = x * scale rounded toward zero to FP16; k = |x * scale - h|
    / (ulp(h) / 256) rounded to nearest (halves to even), with ulp(h) = 2^(max(E, 1) - 25) for h's
    biased exponent E; k = 256 moves h one FP16 value away from zero and k to 0 (beyond FP16's
    largest value, k saturates at 255); the value is (h + sign(h) k ulp(h) / 256) / scale."""
    xs = np.atleast_1d(np.asarray(x, np.float32) * np.float32(scale))
    with np.errstate(over="ignore"):  # beyond FP16's range: inf, cut back to 65504 below
        h = xs.astype(np.float16)  # nearest; then cut toward zero
    over = np.abs(h.astype(np.float32)) > np.abs(xs)
    h[over] = np.nextafter(h[over], np.float16(0))
    r = np.abs(xs - h.astype(np.float32)).astype(np.float64)  # exact
    e = np.maximum((h.view(np.uint16).astype(np.int64) >> 10) & 0x1F, 1)
    step = np.ldexp(1.0, e - 33)
    k = np.rint(r / step)
    hmax = np.float16(65504.0)
    carry = (k == 256) & (np.abs(h) < hmax)
    away = np.where(np.signbit(h), np.float16(-np.inf), np.float16(np.inf))
    h[carry] = np.nextafter(h[carry], away[carry])
    k[carry] = 0
    k = np.minimum(k, 255)
    e = np.maximum((h.view(np.uint16).astype(np.int64) >> 10) & 0x1F, 1)
    step = np.ldexp(1.0, e - 33)
    out = ((h.astype(np.float64) + np.copysign(k * step, h.astype(np.float64))) / scale).astype(np.float32)
    return out.reshape(np.shape(x)) if np.ndim(x) else out[0]
