"""Pin of the oracle's surrogate network: its analytic gradient equals central finite
differences of its forward pass (FP64, exact weights), on every parameter block."""
import numpy as np

from oracle import surrogate as S


def test_oracle_gradient_matches_finite_differences():
    cell, nf, no, C, H, B = 4, 2, 3, 3, 5, 2
    rng = np.random.default_rng(0)
    n = S.n_params(cell, nf, no, C, H)
    p = rng.standard_normal(n) * 0.4
    x = rng.standard_normal((B, 2 * cell ** 3))
    f = rng.standard_normal((B, nf))
    dy = rng.standard_normal((B, no))
    g = S.backward(p, x, f, dy, cell, nf, no, C, H, round_bf16=False)
    idx = rng.choice(n, size=60, replace=False)
    for L in S.layout(cell, nf, no, C, H):          # include the first weight and bias of each layer
        idx = np.concatenate([idx, [L["woff"], L["boff"]]])
    eps = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = eps
        yp, _ = S.forward(p + e, x, f, cell, nf, no, C, H, round_bf16=False)
        ym, _ = S.forward(p - e, x, f, cell, nf, no, C, H, round_bf16=False)
        fd = float(np.sum(dy * (yp - ym)) / (2 * eps))
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_is_nearest_even():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.1415926, 0.0])
    r = S.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0            # exact tie 1 + 2^-8 rounds to even (1.0)
    assert r[2] == 1.0078125                      # above the tie rounds up
    assert abs(r[3] + 3.140625) < 1e-12
    assert r[4] == 0.0
