"""The float32 screen of the neighbour and work-count kernels (host emulation, no GPU).

The kernels decide whether a grid point p lies strictly inside an atom's support sphere (centre T,
radius rc) from float32 offsets relative to the brick centre c, and fall back to the float64 test
when the float32 squared distance lies within m = 4e-6 (2 rc + 4 rad)^2 + 1e-6 rc^2 of rc^2
(rad: the brick's bounding radius).  This checks, with numpy's float32 arithmetic in the kernels'
order, that every decision taken in float32 agrees with the float64 one, on points and centres
drawn next to the sphere's surface at the geometric extremes the kernels allow (|p - c| <= rad,
|T - c| < rc + rad)."""
import numpy as np


def _screen(p, c, T, rc, rad):
    P = (p - c).astype(np.float32)
    t = (T - c).astype(np.float32)
    d = P - t
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
    ext = 2.0 * rc + 4.0 * rad
    m = 4e-6 * ext * ext + 1e-6 * rc * rc
    return r2 < np.float32(rc * rc - m), r2 >= np.float32(rc * rc + m)


def test_float32_screen_never_contradicts_float64():
    rng = np.random.default_rng(0)
    for rc, rad, off in [(7.0, 1.05, 0.0), (6.0, 2.6, 25.0), (0.5, 2.5, -40.0), (12.0, 0.3, 1e3)]:
        n = 200_000
        c = np.full(3, off) + rng.normal(0.0, 1.0, 3)
        u = rng.normal(size=(n, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        p = c + u * rad * rng.uniform(0.0, 1.0, (n, 1))  # points of the brick
        v = rng.normal(size=(n, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        # centres at distance rc (1 + e) from the point, e spread over the shell and beyond it
        e = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-9, -1, n)
        T = p + v * (rc * (1.0 + e))[:, None]
        keep = np.linalg.norm(T - c, axis=1) < rc + rad
        p, T, e = p[keep], T[keep], e[keep]
        inside, outside = _screen(p, c, T, rc, rad)
        r2 = np.sum((p - T) ** 2, axis=1)
        assert np.all(r2[inside] < rc * rc), (rc, rad)
        assert np.all(r2[outside] >= rc * rc), (rc, rad)
        # the shell is thin: points 5 % of rc or more from the surface are decided in float32
        far = np.abs(e) >= 0.05
        if far.any():
            assert np.all((inside | outside)[far]), (rc, rad)
