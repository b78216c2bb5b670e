"""Pins of the oracle's FP64 surrogate network (oracle/mlp.c).

* backpropagation equals FP64 central differences of the loss (rel <= 1e-6);
* the feature map sends the corners of the trained box to +-1;
* a network with all weights zero outputs its output bias, whatever the input;
* with only biases and the last layer set, the output is b4 + W4 silu(b3),
  silu evaluated at points where it has a closed form (silu(0) = 0);
* a chain of single weights carries one input through all three hidden SiLU
  layers to an output: at pre-activations +-ln 3 the result has a closed form,
  and random chains equal the nested composition in 50-digit arithmetic.
"""
import math

import numpy as np


def test_backprop_matches_central_differences(oracle_mod):
    rng = np.random.default_rng(21)
    p = rng.normal(0.0, 0.25, oracle_mod.MLP_PARAMS)
    X = rng.uniform(-1, 1, (6, 4))
    Y = rng.uniform(0, 1, (6, 2))
    loss, g = oracle_mod.mlp_loss_grad(p, X, Y)
    idx = np.concatenate([rng.choice(256, 8, replace=False),               # W1
                          256 + rng.choice(64, 4, replace=False),          # b1
                          320 + rng.choice(4096, 12, replace=False),       # W2
                          4480 + rng.choice(4096, 12, replace=False),      # W3
                          8576 + rng.choice(64, 4, replace=False),         # b3
                          8640 + rng.choice(128, 6, replace=False), [8768, 8769]])
    h = 1e-5
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle_mod.mlp_loss_grad(pp, X, Y)[0] - oracle_mod.mlp_loss_grad(pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3), (i, fd, g[i])


def test_feature_map_box_corners(oracle_mod):
    # no absorption: transmittance 1; opaque (alpha d = 100): transmittance ~ 0;
    # alpha d = ln 2: transmittance 1/2, the middle of the range
    assert np.allclose(oracle_mod.mlp_features(1.0, 780.0, 1.0, 0.010, 0.0), [1, 1, 1, 1], atol=1e-12)
    assert np.allclose(oracle_mod.mlp_features(0.0, 380.0, 0.0, 0.002, 5e4), [-1, -1, -1, -1], atol=1e-12)
    assert np.allclose(oracle_mod.mlp_features(0.25, 580.0, 0.5, 0.006, np.log(2.0) / 0.006), [0, 0, 0, 0],
                       atol=1e-12)
    # the angle enters as sqrt(cos): cos = 1/16 sits a quarter of the way up
    assert abs(oracle_mod.mlp_features(1.0 / 16.0, 580.0, 0.5, 0.006, 1.0)[0] + 0.5) <= 1e-12


def test_feature_transmittance_is_beer_lambert(oracle_mod):
    """x3 is 2 T_int - 1 with T_int the internal transmittance of the slab at
    normal incidence: halving the thickness takes its square root, and for a
    material law alpha = alpha_clear + s dalpha it falls with s as
    exp(-s dalpha d)."""
    for ad in (0.05, 0.7, 3.0):
        t_full = (oracle_mod.mlp_features(0.3, 500.0, 0.2, 0.008, ad / 0.008)[3] + 1) / 2
        t_half = (oracle_mod.mlp_features(0.3, 500.0, 0.2, 0.004, ad / 0.008)[3] + 1) / 2
        assert abs(t_half - np.sqrt(t_full)) <= 1e-12
    ac, da, d = 20.0, 400.0, 0.004
    t0 = (oracle_mod.mlp_features(0.5, 600.0, 0.0, d, ac)[3] + 1) / 2
    for s in (0.25, 0.5, 1.0):
        ts = (oracle_mod.mlp_features(0.5, 600.0, s, d, ac + s * da)[3] + 1) / 2
        assert abs(ts / t0 - np.exp(-s * da * d)) <= 1e-12


def test_constant_networks(oracle_mod):
    p = np.zeros(oracle_mod.MLP_PARAMS)
    p[8768], p[8769] = 0.25, -0.5
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (5, 4))
    assert np.allclose(oracle_mod.mlp_forward(p, X), [[0.25, -0.5]] * 5, atol=0)
    # hidden layers constant: h3 = silu(b3); with b3 = 0 on half the units silu is exactly 0
    p[8576:8576 + 32] = 0.0
    p[8576 + 32:8640] = 2.0
    p[8640:8704] = 1.0            # W4 row 0
    p[8704:8768] = -1.0           # W4 row 1
    s2 = 2.0 / (1.0 + math.exp(-2.0))
    want = np.array([0.25 + 32 * s2, -0.5 - 32 * s2])
    assert np.allclose(oracle_mod.mlp_forward(p, X), [want] * 5, rtol=1e-12)
    loss, g = oracle_mod.mlp_loss_grad(p, X, np.zeros((5, 2)))
    assert abs(loss - (want ** 2).mean()) < 1e-9
    assert np.all(g[:8576] == 0.0)       # nothing reaches the constant layers' weights


def test_served_output_map(oracle_mod):
    """Served (R, T) = exp(y) - 1e-3 clamped at 0: a constant network whose
    output biases are log(v + 1e-3) serves exactly v; outputs below log(1e-3)
    serve 0."""
    p = np.zeros(oracle_mod.MLP_PARAMS, np.float32)
    X = np.random.default_rng(5).uniform(-1, 1, (4, 4))
    for R, T in ((0.25, 0.5), (0.04, 0.9), (1.0, 0.0)):
        p[8768], p[8769] = np.log(R + 1e-3), np.log(T + 1e-3)
        rt = oracle_mod.mlp_rt(p, X)
        # the float32 biases round log(v + 1e-3) to 2^-24 relative
        assert np.allclose(rt, [[R, T]] * 4, rtol=1e-6, atol=1e-9)
    p[8768], p[8769] = np.log(5e-4), np.log(1e-6)
    assert np.array_equal(oracle_mod.mlp_rt(p, X), np.zeros((4, 2)))


def test_feature_film_absorbance_adds_to_the_substrate(oracle_mod):
    """Coating films enter x3 through their Beer-Lambert absorbance: a film of
    absorbance A multiplies the transmittance by exp(-A), exactly as extra
    substrate absorption alpha' d = alpha d + A would."""
    for A in (0.0, 0.3, 1.7):
        a = oracle_mod.mlp_features(0.4, 650.0, 0.7, 0.004, 25.0, A)[3]
        b = oracle_mod.mlp_features(0.4, 650.0, 0.7, 0.004, 25.0 + A / 0.004)[3]
        assert abs(a - b) <= 1e-12
        t0 = (oracle_mod.mlp_features(0.4, 650.0, 0.7, 0.004, 25.0)[3] + 1) / 2
        assert abs((a + 1) / 2 - t0 * np.exp(-A)) <= 1e-12


def _chain_params(units, w, b, b4):
    """A network in which one chain of single nonzero weights carries input
    x[units[0]] through hidden units units[1], units[2], units[3] to output
    units[4]: W1[u1][u0] = w[0], W2[u2][u1] = w[1], W3[u3][u2] = w[2],
    W4[u4][u3] = w[3], the chain's biases b, output biases b4."""
    u0, u1, u2, u3, u4 = units
    p = np.zeros(8770)
    p[0 + 4 * u1 + u0] = w[0]            # W1[64][4]
    p[256 + u1] = b[0]                   # b1
    p[320 + 64 * u2 + u1] = w[1]         # W2[64][64]
    p[4416 + u2] = b[1]                  # b2
    p[4480 + 64 * u3 + u2] = w[2]        # W3[64][64]
    p[8576 + u3] = b[2]                  # b3
    p[8640 + 64 * u4 + u3] = w[3]        # W4[2][64]
    p[8768:8770] = b4
    return p


def test_signal_through_every_layer_closed_form(oracle_mod):
    """A single chain of weights through all four layers, with pre-activations
    placed where SiLU has a closed value: sigma(ln 3) = 3/4, so
    silu(ln 3) = (3/4) ln 3 and silu(-ln 3) = -(1/4) ln 3.

    Layer 1: z1 = x0 + (ln 3 - x0) = ln 3          -> h1 = (3/4) ln 3
    Layer 2: z2 = (4/3) h1 = ln 3                  -> h2 = (3/4) ln 3
    Layer 3: z3 = -(4/3) h2 = -ln 3                -> h3 = -(1/4) ln 3
    Output:  y  = b4 + 4 h3 = b4 - ln 3.

    Dropping the SiLU of any hidden layer, applying one to the output, a
    transposed weight index or a bias taken from the wrong unit changes y."""
    ln3 = math.log(3.0)
    x0 = 0.375
    X = np.array([[0.0, 0.0, x0, 0.0]])
    p = _chain_params((2, 7, 33, 50, 1), (1.0, 4.0 / 3.0, -4.0 / 3.0, 4.0),
                      (ln3 - x0, 0.0, 0.0), (0.125, 0.5))
    y = oracle_mod.mlp_forward(p, X)[0]
    assert abs(y[0] - 0.125) <= 1e-15
    assert abs(y[1] - (0.5 - ln3)) <= 1e-14
    # the other inputs do not reach the chain
    X2 = np.array([[0.9, -0.4, x0, 0.7]])
    assert np.array_equal(oracle_mod.mlp_forward(p, X2)[0], y)


def test_signal_through_every_layer_mpmath(oracle_mod):
    """Random chain weights and biases, five chains summed into both outputs:
    the oracle's forward equals the nested composition
    y = b4 + sum_chains w4 silu(w3 silu(w2 silu(w1 x + b1) + b2) + b3)
    evaluated in 50-digit arithmetic."""
    mpmath = __import__("pytest").importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(77)
    p = np.zeros(8770)
    chains = []
    used = set()
    for c in range(5):
        while True:
            units = (int(rng.integers(4)), int(rng.integers(64)), int(rng.integers(64)), int(rng.integers(64)),
                     c % 2)
            if units[1:4] not in used and len({units[1], units[2], units[3]}) == 3:
                break
        # each hidden unit belongs to one chain only, so the chains do not mix
        if any(u in {v for ch in chains for v in ch[0][1:4]} for u in units[1:4]):
            continue
        used.add(units[1:4])
        w = rng.uniform(-2.0, 2.0, 4)
        b = rng.uniform(-1.0, 1.0, 3)
        q = _chain_params(units, w, b, (0.0, 0.0))
        p += q
        chains.append((units, w, b))
    assert len(chains) >= 3
    p[8768:8770] = (0.3, -0.2)
    X = rng.uniform(-1, 1, (4, 4))

    def silu(z):
        return z / (1 + mpmath.exp(-z))

    got = oracle_mod.mlp_forward(p, X)
    for i in range(X.shape[0]):
        want = [mpmath.mpf(0.3), mpmath.mpf(-0.2)]
        for units, w, b in chains:
            h1 = silu(mpmath.mpf(w[0]) * mpmath.mpf(X[i, units[0]]) + mpmath.mpf(b[0]))
            h2 = silu(mpmath.mpf(w[1]) * h1 + mpmath.mpf(b[1]))
            h3 = silu(mpmath.mpf(w[2]) * h2 + mpmath.mpf(b[2]))
            want[units[4]] += mpmath.mpf(w[3]) * h3
        for o in range(2):
            assert abs(got[i, o] - float(want[o])) <= 1e-14, (i, o, got[i, o], want[o])
