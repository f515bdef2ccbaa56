"""Why the mixed path keeps FP64 origins per body rather than per grid cell.

The mixed contact kernel forms the branch vector from a per-row FP32 reference
vector g (the FP64 branch at the collider run, rounded once) plus the FP32 change e of
both bodies' offsets from their FP64 origins, and takes the contact test and the
penetration from the squared gap s0 - 2 g.e - e.e, s0 = (r1 + r2)^2 - |g|^2 formed in
FP64 at the collider run.  With per-body origins (each body's position at that run)
e is the motion since the run, so every FP32 term is of the size of the gap or of that
motion.  With per-cell origins (the corner of the body's grid cell) the offsets are of
the size of a cell and the FP32 terms carry rounding of the cell's size.

This is a host emulation in numpy float32, in the kernel's operation order, of the
penetration (hence Fn = kn pen) of random contacts of the 1M-sphere compaction's
geometry (log-normal radii, median 1 mm; relative motion since the collider run up to
the Verlet margin, 0.25 mm), against the FP64 penetration of the same positions.  It
needs no GPU and no oracle: it compares two FP32 restatements of one formula against
its FP64 evaluation.  Both variants move the same bytes (a per-row reference vector, a
per-body FP32 offset), so the comparison is on error alone.
"""
import numpy as np

f32, f64 = np.float32, np.float64
MARGIN = 0.25e-3


def _geometry(m, seed=7):
    rng = np.random.default_rng(seed)
    r1 = np.clip(np.exp(np.log(1e-3) + 0.25 * rng.standard_normal(m)), 5e-4, 2e-3)
    r2 = np.clip(np.exp(np.log(1e-3) + 0.25 * rng.standard_normal(m)), 5e-4, 2e-3)
    R = r1 + r2
    p = 10 ** rng.uniform(-6, -2, m)            # penetration / (r1 + r2) now
    n = rng.standard_normal((m, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    x1 = rng.uniform(0, 0.21, (m, 3))            # the cell's side at the dense end
    x2 = x1 + n * (R * (1 - p))[:, None]

    def ball(s):
        u = rng.standard_normal((m, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        return u * (s * rng.uniform(0, 1, m) ** (1 / 3))[:, None]

    xr1, xr2 = x1 - ball(MARGIN / 2), x2 - ball(MARGIN / 2)
    return r1, r2, R, p, x1, x2, xr1, xr2


def _dot(a, b):   # a.x b.x + a.y b.y + a.z b.z in float32, left to right
    return (a[:, 0] * b[:, 0] + a[:, 1] * b[:, 1]) + a[:, 2] * b[:, 2]


def _squared_gap_pen(R, Rf, G64, o1, o2):
    g = G64.astype(f32)
    s0 = (R * R - (G64[:, 0] ** 2 + G64[:, 1] ** 2 + G64[:, 2] ** 2)).astype(f32)
    e = o2.astype(f32) - o1.astype(f32)
    gap2 = s0 - (f32(2) * _dot(g, e) + _dot(e, e))
    d = g + e
    return (gap2 / (Rf + np.sqrt(_dot(d, d)))).astype(f64)


def _errors(m=400_000):
    r1, r2, R, p, x1, x2, xr1, xr2 = _geometry(m)
    exact = R - np.linalg.norm(x2 - x1, axis=1)
    Rf = r1.astype(f32) + r2.astype(f32)
    h = 2 * 2e-3 + 2 * MARGIN                     # a grid cell: 2 r_max + 2 margin
    O1, O2 = np.floor(xr1 / h) * h, np.floor(xr2 / h) * h
    body = _squared_gap_pen(R, Rf, xr2 - xr1, x1 - xr1, x2 - xr2)
    cell = _squared_gap_pen(R, Rf, O2 - O1, x1 - O1, x2 - O2)
    return p, np.abs(body - exact) / exact, np.abs(cell - exact) / exact


def test_per_body_origins_beat_per_cell_origins_at_every_depth():
    p, body, cell = _errors()
    print("\npen/(r1+r2)   median rel. error of Fn: per-body | per-cell;  share above 1e-5")
    for a in range(-6, -2):
        m = (p >= 10.0 ** a) & (p < 10.0 ** (a + 1))
        mb, mc = np.median(body[m]), np.median(cell[m])
        print(f"[1e{a}, 1e{a + 1})   {mb:.2e} | {mc:.2e};  "
              f"{np.mean(body[m] > 1e-5):.1%} | {np.mean(cell[m] > 1e-5):.1%}")
        # the cell-sized FP32 terms cost more than an order of magnitude at every depth
        assert mc > 10 * mb
    # at the depths of a loaded packing (pen/R >= 1e-3) per-body origins meet 1e-5
    deep = p >= 1e-3
    assert np.mean(body[deep] > 1e-5) < 0.01
    assert np.mean(cell[deep] > 1e-5) > 0.5


def test_emulation_reduces_to_fp64_without_rounding():
    """The emulated formula is the penetration: evaluated in FP64 (no FP32 rounding)
    with either origin it matches R - |x2 - x1| to FP64 rounding (a wrong sign or a
    dropped term of the squared gap fails here)."""
    r1, r2, R, p, x1, x2, xr1, xr2 = _geometry(20_000, seed=3)
    exact = R - np.linalg.norm(x2 - x1, axis=1)
    h = 2 * 2e-3 + 2 * MARGIN
    O1, O2 = np.floor(xr1 / h) * h, np.floor(xr2 / h) * h
    for G, o1, o2 in ((xr2 - xr1, x1 - xr1, x2 - xr2), (O2 - O1, x1 - O1, x2 - O2)):
        s0 = R * R - np.sum(G * G, axis=1)
        e = o2 - o1
        gap2 = s0 - (2 * np.sum(G * e, axis=1) + np.sum(e * e, axis=1))
        pen = gap2 / (R + np.linalg.norm(G + e, axis=1))
        assert np.max(np.abs(pen - exact) / exact) < 1e-6
