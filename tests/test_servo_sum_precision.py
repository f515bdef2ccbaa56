"""The error of the stress servo's sums in mixed precision.  The GPU forms, per real
contact, the products sigma_aa V: F_a (-l n_a) and K_a V: kn (l n_a)^2 from FP32
operands in FP32, sums them in FP32 over runs of 8 rows, and adds the run sums in
FP64.  This emulates that arithmetic with numpy's FP32 (every product and sum
rounded, which has at least as many roundings as the kernel's fused multiply-adds)
and checks the bounds the kernel states: a run sum of the stiffness terms (all
positive) within (8 + 3) units of FP32 machine epsilon relative, a run sum of the
stress terms within that many units of the sum of its terms' magnitudes, and the
whole sums of a million contacts within 1e-6 relative of the FP64 sums of the same
operands.  Inputs: a dense packing's contacts (branch length 2 mm +- 20%, unit
normals, normal forces log-normal around 1 N, shear forces up to 0.5 of them,
kn log-uniform in [1e4, 1e6] N/m)."""
import numpy as np

RUN = 8
EPS32 = 2.0 ** -23


def _contacts(n, seed):
    rng = np.random.default_rng(seed)
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    l = 2e-3 * rng.uniform(0.8, 1.2, n)
    d1 = l * rng.uniform(0.4, 0.6, n)
    d2 = l - d1
    fn = np.exp(rng.normal(0.0, 1.0, n))
    ft = rng.normal(size=(n, 3))
    ft -= np.sum(ft * nrm, axis=1)[:, None] * nrm
    ft *= (0.5 * fn * rng.uniform(0, 1, n) / np.maximum(np.linalg.norm(ft, axis=1), 1e-300))[:, None]
    F = -fn[:, None] * nrm + ft
    kn = 10.0 ** rng.uniform(4, 6, n)
    f32 = np.float32
    return (F.astype(f32), nrm.astype(f32), d1.astype(f32), d2.astype(f32), kn.astype(f32))


def _fp32_runs(F, nrm, d1, d2, kn):
    """Run sums in FP32, (runs, 6), in the kernel's operation order."""
    n = len(kn)
    l = (d1 + d2).astype(np.float32)                  # FP32 sum of the two branch lengths
    bl = (l[:, None] * nrm).astype(np.float32)
    s = (F * bl).astype(np.float32)
    k = (kn[:, None] * (bl * bl).astype(np.float32)).astype(np.float32)
    terms = np.concatenate([-s, k], axis=1).reshape(n // RUN, RUN, 6)
    acc = np.zeros((n // RUN, 6), dtype=np.float32)
    for j in range(RUN):
        acc = (acc + terms[:, j]).astype(np.float32)
    return acc


def _fp64_terms(F, nrm, d1, d2, kn):
    l = d1.astype(np.float64) + d2.astype(np.float64)
    bl = l[:, None] * nrm.astype(np.float64)
    s = F.astype(np.float64) * bl
    k = kn.astype(np.float64)[:, None] * bl * bl
    return np.concatenate([-s, k], axis=1)


def test_run_sums_within_stated_bound():
    F, nrm, d1, d2, kn = _contacts(RUN * 20000, 5)
    runs = _fp32_runs(F, nrm, d1, d2, kn).astype(np.float64)
    exact = _fp64_terms(F, nrm, d1, d2, kn).reshape(-1, RUN, 6)
    mag = np.abs(exact).sum(axis=1)
    err = np.abs(runs - exact.sum(axis=1))
    bound = (RUN + 3) * EPS32 * mag
    assert np.all(err <= bound), float(np.max(err / bound))
    # stiffness runs: relative to the sum itself (all terms positive)
    assert np.all(err[:, 3:] <= (RUN + 3) * EPS32 * exact.sum(axis=1)[:, 3:])


def test_whole_sums_of_a_million_contacts():
    F, nrm, d1, d2, kn = _contacts(RUN * 125000, 6)
    total32 = _fp32_runs(F, nrm, d1, d2, kn).astype(np.float64).sum(axis=0)
    total64 = _fp64_terms(F, nrm, d1, d2, kn).sum(axis=0)
    assert np.all(total64[:3] > 0) and np.all(total64[3:] > 0)   # compression, stiffness
    assert np.all(np.abs(total32 / total64 - 1) < 1e-6), total32 / total64 - 1


def test_a_planted_fp32_total_fails():
    """The same check on one FP32 accumulator over all rows (no FP64 across runs)
    is what the run length guards against: its error is far larger."""
    F, nrm, d1, d2, kn = _contacts(RUN * 125000, 6)
    runs = _fp32_runs(F, nrm, d1, d2, kn)
    acc = np.zeros(6, dtype=np.float32)
    for r in runs:
        acc = (acc + r).astype(np.float32)
    total64 = _fp64_terms(F, nrm, d1, d2, kn).sum(axis=0)
    assert np.max(np.abs(acc.astype(np.float64) / total64 - 1)) > 1e-6
