"""Surrogate network on the GPU (hand-written forward / backward / Adam kernels) against the FP64
oracle with the same BF16-rounded weights: forward within 1e-5, parameter gradients within 1e-4
(relative, per layer block) -- FP32 accumulation over at most a few thousand terms; and training
by the library's own kernels reduces the loss of a teacher-student regression."""
import numpy as np
import pytest

from oracle import surrogate as S

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


@pytest.mark.parametrize("cell,C,H,nf,no,B", [(8, 4, 16, 3, 7, 3), (16, 6, 12, 5, 9, 2)])
def test_forward_backward_match_oracle(P, cell, C, H, nf, no, B):
    net = P.Surrogate(cell, nf, no, channels=C, hidden=H, seed=3)
    assert net.n_params == S.n_params(cell, nf, no, C, H)
    rng = np.random.default_rng(1)
    p = (rng.standard_normal(net.n_params) * 0.3).astype(np.float32)
    net.set_params(p)
    x = rng.standard_normal((B, 2 * cell ** 3)).astype(np.float32)
    f = rng.standard_normal((B, nf)).astype(np.float32)
    dy = rng.standard_normal((B, no)).astype(np.float32)
    xd, fd, dyd = (torch.tensor(a, device="cuda") for a in (x, f, dy))
    y = torch.zeros((B, no), device="cuda")
    net.forward(xd, fd, y)
    g = torch.zeros(net.n_params, device="cuda")
    net.backward(xd, fd, dyd, g)
    torch.cuda.synchronize()
    yr, _ = S.forward(p.astype(np.float64), x, f, cell, nf, no, C, H)
    gr = S.backward(p.astype(np.float64), x, f, dy, cell, nf, no, C, H)
    assert np.linalg.norm(y.cpu().numpy() - yr) <= 1e-5 * np.linalg.norm(yr)
    gg = g.cpu().numpy().astype(np.float64)
    for L in S.layout(cell, nf, no, C, H):
        for a, b in ((L["woff"], L["boff"]), (L["boff"], L["boff"] + L["cout"])):
            ref = gr[a:b]
            assert np.linalg.norm(gg[a:b] - ref) <= 1e-4 * max(np.linalg.norm(ref), 1e-12), (L, a)


def test_training_reduces_loss(P):
    cell, C, H, nf, no, B = 8, 8, 32, 4, 20, 64
    rng = np.random.default_rng(2)
    teacher = rng.standard_normal(S.n_params(cell, nf, no, C, H)) * 0.25
    x = rng.standard_normal((B, 2 * cell ** 3)).astype(np.float32)
    f = rng.standard_normal((B, nf)).astype(np.float32)
    t, _ = S.forward(teacher, x, f, cell, nf, no, C, H, round_bf16=False)
    net = P.Surrogate(cell, nf, no, channels=C, hidden=H, seed=9)
    xd, fd, td = (torch.tensor(a, device="cuda", dtype=torch.float32) for a in (x, f, t))
    loss = torch.zeros(1, device="cuda")
    hist = []
    for it in range(400):
        net.train_step(xd, fd, td, 3e-3, loss)
        if it in (0, 399):
            torch.cuda.synchronize()
            hist.append(float(loss.item()))
    assert hist[1] < 0.05 * hist[0], hist
