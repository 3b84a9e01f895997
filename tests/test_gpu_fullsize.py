"""GPU parity at the full 64^3 / 512-box size, in the launch configuration bench.py times.

At this size the CUDA path takes branches the small parity cases never reach: four right-hand sides
per CTA of the banded F-apply (512 boxes on one shape's shared factor record), the 69-block-column
factorisation of 8^3 boxes on a thread-block cluster, and the tensor-core dual Schur apply over four
128-row tiles.  The oracle's outputs for these inputs are stored, sampled at seeded indices (every
k-th of 4096 per vector, k the record's sample_stride), in tests/golden/cube64_parity_record.json, written by tests/golden/make_cube64_parity_record.py
from oracle/ only; the test regenerates the seeded inputs and first checks them against the record's
fingerprints.

Tolerances as in the small parity cases: operator applies in FP64 to 1e-10 (F, K^+) and 1e-11
(P_N, B K B^T, N) of the vector's largest entry; dual solutions at eps_PCGP = 1e-12 to 1e-9; plastic
flags exactly, except within |Phi| <= 1e-8 sigma_y of the yield surface.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines only
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1205_1926_gb300 as T  # noqa: E402

REC_PATH = os.path.join(os.path.dirname(__file__), "golden", "cube64_parity_record.json")


@pytest.fixture(scope="module")
def rec():
    with open(REC_PATH) as fh:
        return json.load(fh)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def zeros(n, dtype=torch.float64):
    return torch.zeros(int(n), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def check_fingerprint(v, fp):
    assert v.size == fp["n"]
    assert [float(a) for a in v[:3]] == fp["head"] and [float(a) for a in v[-3:]] == fp["tail"]
    assert abs(float(v.sum()) - fp["sum"]) <= 1e-12 * max(1.0, abs(fp["sum"])) * np.sqrt(v.size)


def inputs(rec):
    s = rec["seeds"]
    idx_m = W.seeded_indices(rec["n_mult"], rec["n_samples"], s["mult_idx"])
    idx_d = W.seeded_indices(rec["n_dof"], rec["n_samples"], s["dof_idx"])
    idx_g = W.seeded_indices(rec["n_gp"], rec["n_samples"], s["gp_idx"])
    assert [int(idx_m.sum()), int(idx_d.sum()), int(idx_g.sum())] == rec["inputs"]["idx_sums"]
    k = rec.get("sample_stride", 1)         # the record keeps every k-th sampled value
    idx_m, idx_d, idx_g = idx_m[::k], idx_d[::k], idx_g[::k]
    x = W.seeded_vector(rec["n_mult"], seed=s["x"])
    v = W.seeded_vector(rec["n_dof"], seed=s["v"])
    du, hot = W.seeded_partly_plastic_increment(W.CUBE64, s["du"], s["n_hot"])
    check_fingerprint(x, rec["inputs"]["x"])
    check_fingerprint(v, rec["inputs"]["v"])
    check_fingerprint(du, rec["inputs"]["du"])
    assert hot == rec["inputs"]["hot"]
    return idx_m, idx_d, idx_g, x, v, du


def assert_sampled(y, idx, ref, tol, what):
    """Sampled entries within tol of the vector's largest entry, and its norm within tol."""
    vals = np.asarray(ref["values"])
    err = np.abs(y[idx] - vals).max()
    assert err <= tol * ref["max_abs"], (what, err / ref["max_abs"])
    assert abs(np.linalg.norm(y) - ref["norm"]) <= tol * ref["norm"], (what, np.linalg.norm(y), ref["norm"])


@pytest.fixture(scope="module")
def ctx64():
    c = T.Context(W.CUBE64)
    yield c
    c.close()


@pytest.mark.parametrize("part", ["ops_elastic", "ops_partly_plastic"])
def test_cube64_operators_elementwise(rec, ctx64, part):
    """F, P_N, B K B^T, N and K^+ at 64^3 against the oracle; the FP32 inner F-apply of the mixed
    mode (tensor-core Schur apply over 4 M-tiles, FP32 banded solves for the plastic boxes) against
    the same oracle values to FP32 accuracy."""
    idx_m, idx_d, _, x, v, du = inputs(rec)
    ctx = ctx64
    s = ctx.sizes
    r = rec[part]
    zs = zeros(6 * s["n_gp"])
    ctx.set_state(u=zeros(s["n_dof"]), sigma=zs, kappa=zeros(s["n_gp"]))
    ctx.set_precision(False)
    inc = du if part == "ops_partly_plastic" else np.zeros(s["n_dof"])
    ctx.assemble_tangent(dev(inc), zeros(s["n_dof"]), zeros(s["n_dof"]))
    m = s["n_mult"]
    y = zeros(m)
    dx = dev(x)
    ctx.apply("F", dx, y)
    yF = host(y)
    assert_sampled(yF, idx_m, r["F"], 1e-10, "F")
    ctx.apply("projector", dx, y)
    assert_sampled(host(y), idx_m, r["projector"], 1e-11, "P")
    ctx.apply("precond", dx, y)
    assert_sampled(host(y), idx_m, r["precond"], 1e-11, "precond")
    yN = zeros(s["n_coarse"])
    ctx.apply("N", dx, yN)
    ref = np.asarray(r["N"])
    assert np.abs(host(yN) - ref).max() <= 1e-11 * np.abs(ref).max()
    yk = zeros(s["n_dof"])
    ctx.apply("kdag", dev(v), yk)
    assert_sampled(host(yk), idx_d, r["kdag"], 1e-10, "kdag")
    ctx.set_precision(True, 1e-4)
    ctx.apply("F32", dx, y)
    y32 = host(y)
    assert np.isfinite(y32).all()
    assert_sampled(y32, idx_m, r["F"], 2e-5, "F32")
    assert np.linalg.norm(y32 - yF) <= 1e-5 * np.linalg.norm(yF)
    ctx.set_precision(False)


@pytest.mark.parametrize("mixed", [False, True])
def test_cube64_dual_solve_elementwise(rec, ctx64, mixed):
    """Algorithm 3 at eps_PCGP = 1e-12 on the partly plastic 64^3 tangent (48 boxes on own factors,
    464 on the shared one): u and lambda against the oracle, the FP64 iteration count within one; the
    mixed mode (FP64-refined, FP32 inner operators) reaches the same solution."""
    idx_m, idx_d, _, x, v, du = inputs(rec)
    ctx = ctx64
    s = ctx.sizes
    r = rec["dual_solve"]
    ctx.set_state(u=zeros(s["n_dof"]), sigma=zeros(6 * s["n_gp"]), kappa=zeros(s["n_gp"]))
    ctx.set_precision(mixed, 1e-4)
    df = zeros(s["n_dof"])
    ctx.traction_load(tuple(r["traction"]), df)
    f = zeros(s["n_dof"])
    ctx.assemble_tangent(dev(du), df, f)
    u, lam = zeros(s["n_dof"]), zeros(s["n_mult"])
    info = ctx.dual_pcg(f, u, lam, rtol=r["rtol"], maxit=5000)
    assert_sampled(host(u), idx_d, r["u"], 1e-9, "u")
    assert_sampled(host(lam), idx_m, r["lam"], 1e-9, "lambda")
    if not mixed:
        assert abs(info["iterations"] - r["iterations"]) <= 1
    ctx.set_precision(False)


def test_cube64_plastic_load_step_elementwise(rec):
    """One load step of Algorithm 4 from the zero state to 1.5 t_y at (eps_Newton, eps_PCGP) =
    (1e-10, 1e-11) (at this size the FP64 dual residual of the full-load step stalls above 1e-12, in the
    oracle as on the GPU): Newton and PCGP counts, u and the committed kappa and sigma_13 at sampled
    points, and the plastic Gauss points exactly, except those within |Phi| <= 1e-8 sigma_y of the
    yield surface at the commit."""
    _, idx_d, idx_g, _, _, _ = inputs(rec)
    r = rec["plastic_step"]
    w = W.CUBE64
    ctx = T.Context(w)
    s = ctx.sizes
    t_y = ctx.first_yield_traction(w.traction_dir, rtol=1e-10)
    assert abs(t_y - r["t_y"]) <= 1e-9 * r["t_y"]
    df = zeros(s["n_dof"])
    ctx.traction_load(tuple(r["load_fraction"] * r["t_y"] * c for c in w.traction_dir), df)
    info = ctx.time_step(df, r["newton_tol"], r["pcg_rtol"], 30, 5000)
    assert info["converged"] and info["criterion"][0] == 1.0
    assert abs(info["newton"] - r["newton"]) <= 1, (info["newton"], r["newton"])
    n_cmp = min(info["newton"], r["newton"])
    assert all(abs(a - b) <= 1 for a, b in zip(info["pcg"][:n_cmp], r["pcg"][:n_cmp])), (info["pcg"], r["pcg"])
    n_gp = s["n_gp"]
    u, sig, kap = zeros(s["n_dof"]), zeros(6 * n_gp), zeros(n_gp)
    ctx.get_state(u, sig, kap)
    u, sig, kap = host(u), host(sig).reshape(6, n_gp), host(kap)
    assert_sampled(u, idx_d, r["u"], 1e-9, "u")
    assert_sampled(kap, idx_g, r["kappa"], 1e-7, "kappa")
    assert_sampled(sig[5], idx_g, r["sigma_xz"], 1e-8, "sigma_13")
    plastic = np.zeros(n_gp, dtype=bool)
    plastic[np.asarray(r["plastic_idx"], dtype=np.int64)] = True
    band = np.zeros(n_gp, dtype=bool)
    band[np.asarray(r["band_idx"], dtype=np.int64)] = True
    assert plastic.sum() > 0 and info["plastic_committed"] > 0
    np.testing.assert_array_equal((kap > 0)[~band], plastic[~band])
    ctx.close()
