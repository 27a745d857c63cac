"""GPU parity of the learned-closure MLP kernels (BF16 tensor cores, FP32
accumulation) against the FP64 oracle: forward, gradients, AdamW, training."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS = [67, 256, 256, 256, 256, 3]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _closure(members=2, seed=3):
    from paper_2512_13267_gb300 import lhmm as lh
    c = lh.Closure(members=members, in_dim=67, hidden=256, n_hidden=4, out_dim=3, seed=seed)
    c.set_normalization(np.zeros(67), np.ones(67), np.ones(3))
    return c


def _bf16(a):
    """Round float64 values to the nearest bfloat16 (round half to even)."""
    f = np.asarray(a, np.float32).view(np.uint32)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def test_forward_matches_oracle_within_bf16_rounding(parity_report):
    c = _closure()
    rng = np.random.default_rng(0)
    X = rng.normal(size=(100, 67))
    Y = c.forward_members(torch.from_numpy(X.astype(np.float32)).cuda())
    for m in range(2):
        p = c.get_params(m).astype(np.float64)
        ref = O.mlp_forward(DIMS, p, X.astype(np.float32).astype(np.float64))
        err = np.abs(Y[m] - ref).max()
        # BF16 operands (8-bit significand) through five layers: a few 1e-3 of
        # the output scale; an indexing or layout mistake is O(1)
        assert err <= 3e-2 * np.abs(ref).max(), (m, err, np.abs(ref).max())
        assert np.corrcoef(Y[m].ravel(), ref.ravel())[0, 1] > 0.999
        # with the weights and inputs rounded to BF16 in the oracle the bound tightens
        ref_b = O.mlp_forward(DIMS, _bf16(p), _bf16(X))
        assert np.abs(Y[m] - ref_b).max() <= 0.5 * err + 1e-2 * np.abs(ref).max()
        parity_report("MLP forward (BF16 tensor cores), member %d" % m,
                      err / np.abs(ref).max(), 3e-2, "max |dy| / max |y|")
    c.close()


def test_gradient_matches_oracle(parity_report):
    c = _closure(members=2, seed=5)
    rng = np.random.default_rng(1)
    B = 64
    X = rng.normal(size=(B, 67)).astype(np.float32)
    T = rng.normal(size=(B, 3)).astype(np.float32)
    c.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), B, lr=0.0)
    for m in range(2):
        g = c.get_grad(m).astype(np.float64)
        p = c.get_params(m).astype(np.float64)
        loss, ref = O.mlp_loss_grad(DIMS, p, X.astype(np.float64), T.astype(np.float64))
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
        assert rel < 0.05 and cos > 0.998, (m, rel, cos)
        parity_report("MLP loss gradient, member %d" % m, rel, 0.05, "|dg| / |g| (L2)")
    c.close()


def test_adamw_update_matches_oracle_step(parity_report):
    c = _closure(members=1, seed=9)
    rng = np.random.default_rng(2)
    B = 96
    X = torch.from_numpy(rng.normal(size=(B, 67)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(B, 3)).astype(np.float32)).cuda()
    p0 = c.get_params(0).astype(np.float64)
    c.train_step(X, T, B, lr=1e-3, weight_decay=0.0)
    p1 = c.get_params(0).astype(np.float64)
    g = c.get_grad(0).astype(np.float64)
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    exp = p0.copy()
    O.adamw_step(exp, g, m, v, 1e-3, 0.9, 0.999, 1e-8, 0.0, 1)
    assert np.abs(p1 - exp).max() <= 1e-6 + 1e-5 * np.abs(exp).max()
    parity_report("AdamW step", np.abs(p1 - exp).max(), 1e-6 + 1e-5 * np.abs(exp).max(),
                  "max |dp|")
    c.close()


def test_training_reduces_loss_for_every_member():
    c = _closure(members=5, seed=11)
    rng = np.random.default_rng(3)
    N, B = 4096, 256
    X = rng.normal(size=(N, 67)).astype(np.float32)
    T = np.stack([0.5 * X[:, 0] - 0.3 * X[:, 5], np.sin(X[:, 2]), X[:, 1] * X[:, 3] * 0.2],
                 axis=1).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    loss = torch.zeros(5, dtype=torch.float32, device="cuda")
    first = None
    for step in range(300):
        rows = torch.from_numpy(rng.integers(0, N, size=(5, B)).astype(np.int32)).cuda()
        c.train_step(Xd, Td, B, lr=1e-3, weight_decay=1e-4, rows_dev=rows, loss_dev=loss)
        if step == 0:
            first = loss.cpu().numpy().copy()
    last = loss.cpu().numpy()
    assert np.all(last < 0.2 * first), (first, last)
    c.close()


def test_ensemble_mean_and_spread():
    c = _closure(members=5, seed=13)
    c.set_normalization(np.zeros(67), np.ones(67), np.array([2.0, 0.5, 3.0]))
    rng = np.random.default_rng(4)
    X = torch.from_numpy(rng.normal(size=(333, 67)).astype(np.float32)).cuda()
    mean = torch.zeros((333, 3), dtype=torch.float32, device="cuda")
    spread = torch.zeros(333, dtype=torch.float32, device="cuda")
    c.infer(X, mean, spread)
    Y = c.forward_members(X) * np.array([2.0, 0.5, 3.0])
    assert np.allclose(mean.cpu().numpy(), Y.mean(axis=0), rtol=1e-5, atol=1e-5)
    sd = np.sqrt(((Y - Y.mean(axis=0)) ** 2).sum(axis=2).sum(axis=0) / 4)
    assert np.allclose(spread.cpu().numpy(), sd, rtol=1e-4, atol=1e-5)
    c.close()


def test_calibration_folds_linear_map_into_output_layer():
    from paper_2512_13267_gb300 import closure as CL
    c = _closure(members=3, seed=17)
    scale = np.array([2.0, 0.5, 3.0], np.float32)
    c.set_normalization(np.zeros(67), np.ones(67), scale)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(512, 67)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    P = c.forward_members(Xd).mean(axis=0) * scale
    T = (np.array([1.5, -0.7, 2.0]) * P + np.array([0.3, 0.1, -0.2])).astype(np.float32)
    before = [c.get_params(m).astype(np.float64) for m in range(3)]
    a, b = CL.calibrate(c, X, T, scale)
    assert np.allclose(a, [1.5, -0.7, 2.0], rtol=1e-3) and np.allclose(b, [0.3, 0.1, -0.2], atol=1e-3)
    # the fold through the FP64 oracle network: every member's folded output
    # is a y + c / scale of its output before (the map is linear in the last
    # layer, so this holds to the FP32 rounding of the stored parameters)
    Xs = X[:64].astype(np.float64)
    for m in range(3):
        y0 = O.mlp_forward(DIMS, before[m], Xs)
        y1 = O.mlp_forward(DIMS, c.get_params(m).astype(np.float64), Xs)
        assert np.allclose(y1, a * y0 + b / scale, rtol=1e-5, atol=1e-6 * np.abs(y0).max())
    mean = torch.zeros((512, 3), dtype=torch.float32, device="cuda")
    spread = torch.zeros(512, dtype=torch.float32, device="cuda")
    c.infer(Xd, mean, spread)
    assert np.allclose(mean.cpu().numpy(), T, rtol=2e-3, atol=2e-3 * np.abs(T).max())
    c.close()


@pytest.mark.parametrize("rows", [96, 160, 4096])
def test_tensor_core_path_matches_mma_sync_path(rows, parity_report):
    # the tcgen05 products (accumulator in tensor memory, TMA-staged operands)
    # against the mma.sync products on the same BF16 operands: both accumulate
    # in FP32, so outputs differ only by the order of the sums (and the BF16
    # rounding of hidden activations that this can flip); gradients likewise.
    # rows = 96 and 160 leave a partial 128-row tile.
    c = _closure(members=3, seed=7)
    rng = np.random.default_rng(rows)
    X = torch.from_numpy(rng.normal(size=(rows, 67)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(rows, 3)).astype(np.float32)).cuda()
    out, grads = {}, {}
    for path in (0, 1):
        c.set_gemm(path)
        out[path] = c.forward_members(X)
        c.train_step(X, T, rows, lr=0.0)
        c.sync()
        grads[path] = [c.get_grad(m).astype(np.float64) for m in range(3)]
    y0, y1 = out[0], out[1]
    err = np.abs(y1 - y0).max() / np.abs(y0).max()
    assert err <= 2e-3, err
    parity_report("tcgen05 vs mma.sync forward, %d rows" % rows, err, 2e-3, "max |dy| / max |y|")
    for m in range(3):
        g0, g1 = grads[0][m], grads[1][m]
        rel = np.linalg.norm(g1 - g0) / np.linalg.norm(g0)
        assert rel <= 1e-2, (m, rel)
    parity_report("tcgen05 vs mma.sync gradient, %d rows" % rows, rel, 1e-2, "|dg| / |g| (L2)")
    c.close()
