"""The cost model's GPU kernels: gradients against the FP64 reference MLP,
deterministic training, checkpoint round trip."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _model(seed=3, n_in=24, h=128):
    from paper_1906_08687_gb300.lmf import Mlp
    return Mlp(n_in, h, seed)


def test_gradient_matches_fp64_reference():
    import torch
    rng = np.random.default_rng(0)
    m = _model()
    p = m.get_params().astype(np.float64)
    B = 64
    x = (rng.standard_normal((B, 24)) * 2 + 1).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    mean = x.mean(axis=0).astype(np.float32)
    std = (x.std(axis=0) + 0.5).astype(np.float32)
    m.set_norm(mean, std, 0.0, 1.0)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    g = torch.zeros(m.n_params, dtype=torch.float32, device='cuda')
    loss = m.grad(xd.data_ptr(), td.data_ptr(), B, g.data_ptr())
    want_loss, want = ref.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64),
                                        mean.astype(np.float64), std.astype(np.float64), 24, 128)
    got = g.cpu().numpy().astype(np.float64)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss)
    scale = np.abs(want).max()
    np.testing.assert_allclose(got, want, rtol=2e-3, atol=1e-5 * scale)
    # prediction matches the reference forward pass
    y = torch.zeros(B, dtype=torch.float32, device='cuda')
    m.forward(xd.data_ptr(), B, y.data_ptr())
    yr, _ = ref.forward(p, x.astype(np.float64), mean, std, 24, 128)
    np.testing.assert_allclose(y.cpu().numpy(), yr, rtol=1e-4, atol=1e-4)
    m.close()


def test_training_deterministic_and_decreasing():
    import torch
    rng = np.random.default_rng(1)
    X = rng.standard_normal((512, 24)).astype(np.float32)
    w = rng.standard_normal(24).astype(np.float32)
    y = np.tanh(X @ w / 4).astype(np.float32)
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    runs = []
    for _ in range(2):
        m = _model(seed=5)
        m.set_norm(np.zeros(24, np.float32), np.ones(24, np.float32), 0.0, 1.0)
        losses = [m.train_step(xd.data_ptr(), yd.data_ptr(), 512, 1e-3) for _ in range(200)]
        runs.append((m.get_params(), losses))
        m.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.mean(runs[0][1][-20:]) < 0.3 * np.mean(runs[0][1][:5])


def test_checkpoint_round_trip(tmp_path):
    from paper_1906_08687_gb300 import costmodel
    m = _model(seed=9)
    m.norm = (np.zeros(24, np.float32), np.ones(24, np.float32), 0.5, 2.0)
    m.set_norm(*m.norm)
    costmodel.save(m, str(tmp_path / 'cm'), meta={'note': 'test'})
    m2 = costmodel.load(str(tmp_path / 'cm'))
    assert np.array_equal(m.get_params(), m2.get_params())
    f = np.random.default_rng(2).standard_normal((7, 24)).astype(np.float32)
    assert np.array_equal(costmodel.predict(m, f), costmodel.predict(m2, f))
