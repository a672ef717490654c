"""Pin of the oracle's bf16 rounding against torch's bf16 conversion (a library routine).  CPU only."""
import numpy as np
import torch

from oracle import encode, mlp, precision


def test_bf16_round_matches_torch():
    r = np.random.default_rng(0)
    x = np.concatenate([r.standard_normal(100000).astype(np.float32) * 10.0 ** r.integers(-30, 30, 100000),
                        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38, 1e-40, np.inf, -np.inf], np.float32)])
    # exact ties: low 16 bits = 0x8000, both even and odd upper halves
    ties = (r.integers(0, 2 ** 15, 2000, dtype=np.uint32) << 16 | 0x8000).astype(np.uint32).view(np.float32)
    x = np.concatenate([x, ties[np.isfinite(ties)]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = precision.bf16_round(x)
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------- where the emulation rounds
# One level of 2 x 2 x 2 x 1 vertices (8 rows, F = 1): at u = (0, 0, 0, 0) the encoding is the table
# value of vertex 0, at u = (0.25, 0, 0, 0) it is 0.75 T[0] + 0.25 T[1].  bf16 keeps 8 significant
# bits, so on [1, 2) its values are the multiples of 2^-7; a float32 value 1 + k 2^-8 with k odd is a
# tie and rounds to the neighbour whose last mantissa bit is 0.
_E = 2.0 ** -8
_ONE_LEVEL = [[2, 2, 2, 1]]


def _one_neuron(table0, W1, b1, Wo, bo, ux=0.0, table1=1.0, hidden=None):
    table = np.full((8, 1), 1.0)
    table[0, 0], table[1, 0] = table0, table1
    if hidden is None:
        params, dims = [W1, b1, Wo, bo], [1, 1, 1]
    else:
        W2, b2 = hidden
        params, dims = [W1, b1, W2, b2, Wo, bo], [1, 1, 1, 1]
    params = np.array(params, np.float32).astype(np.float64)
    c = np.array([[ux, 0.0, 0.0, 0.0]], np.float32)
    return precision.forward_bf16(_ONE_LEVEL, [0], table.astype(np.float32), params, dims, c)[0]


def test_table_values_are_rounded():
    # T[0] = 1 + 2^-8 is a tie between 1 (even) and 1 + 2^-7: bf16 gives 1, so y = 1 (not 1 + 2^-8)
    assert _one_neuron(1 + _E, 1.0, 0.0, 1.0, 0.0) == 1.0


def test_interpolated_layer_input_is_rounded():
    # bf16 table values 1 and 1 + 2^-6 interpolated at w_x = 1/4 give 1 + 2^-8 exactly, a tie: the
    # first layer sees 1
    assert _one_neuron(1.0, 1.0, 0.0, 1.0, 0.0, ux=0.25, table1=1 + 4 * _E) == 1.0
    # without the table rounding the same point would read 1 + 1.25 2^-8 -> 1 + 2^-7: T[1] = 1 + 5 2^-8
    # rounds (tie, to even) to 1 + 2^-6 first, so the result stays 1
    assert _one_neuron(1.0, 1.0, 0.0, 1.0, 0.0, ux=0.25, table1=1 + 5 * _E) == 1.0


def test_first_layer_weights_are_rounded():
    # W1 = 1 + 3 2^-8 is a tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even): bf16 gives 1 + 2^-6
    assert _one_neuron(1.0, 1 + 3 * _E, 0.0, 1.0, 0.0) == 1 + 4 * _E


def test_hidden_bias_stays_float32():
    # b1 = 2^-8 (1 + 2^-12) would round to 2^-8 in bf16; kept in float32, z = 1 + 2^-8 + 2^-20 lies just
    # above the tie and the output layer's input rounds up to 1 + 2^-7 (a rounded bias would give the
    # tie 1 + 2^-8 and round down to 1)
    assert _one_neuron(1.0, 1.0, _E * (1 + 2.0 ** -12), 1.0, 0.0) == 1 + 2 * _E


def test_output_layer_input_is_rounded():
    # z = 1 + 2^-8 is a tie: the output layer sees 1, so y = 1 (not 1 + 2^-8)
    assert _one_neuron(1.0, 1.0, _E, 1.0, 0.0) == 1.0


def test_output_weights_are_rounded_and_output_bias_is_not():
    assert _one_neuron(1.0, 1.0, 0.0, 1 + 3 * _E, 0.0) == 1 + 4 * _E
    bo = np.float32(0.1)
    assert _one_neuron(1.0, 1.0, 0.0, 1.0, bo) == 1.0 + float(bo)   # bf16(0.1) would be 0.10009765625


def test_relu_and_inner_hidden_layer_rounding():
    # ReLU of a negative pre-activation: the output layer sees 0 and y is the output bias
    assert _one_neuron(1.0, -1.0, 0.0, 1.0, 0.25) == 0.25
    # two hidden layers: z1 = 1 + 2^-8 rounds to 1 before layer 2; z2 = 1 + 2^-8 again rounds to 1.
    # Without the rounding between the hidden layers, z2 = 1 + 2^-7 (exact) and y = 1 + 2^-7.
    assert _one_neuron(1.0, 1.0, _E, 1.0, 0.0, hidden=(1.0, _E)) == 1.0


def test_exact_when_every_value_is_bf16():
    """Integer table values at grid vertices, weights in {-1, 0, 1}, integer biases: every layer input
    is a small integer, exactly a bf16 value, so the emulation must equal the float64 MLP exactly."""
    r = np.random.default_rng(3)
    levels = [[2, 2, 2, 2], [3, 3, 3, 2]]
    from oracle import schedule
    bases, rows = schedule.bases(levels)
    F = 2
    dims = [len(levels) * F, 8, 8, 1]
    table = r.integers(-4, 5, (rows, F)).astype(np.float32)
    params = np.concatenate([np.concatenate([r.integers(-1, 2, dims[k] * dims[k + 1]),
                                             r.integers(-2, 3, dims[k + 1])]) for k in range(len(dims) - 1)])
    params = params.astype(np.float64)
    c = r.integers(0, 2, (500, 4)).astype(np.float32)                  # vertices of both levels
    ref = mlp.forward(params, dims, encode.encode(levels, bases, c, table.astype(np.float64)))[0]
    assert np.abs(ref).max() < 200 and np.abs(ref).max() > 0
    got = precision.forward_bf16(levels, bases, table, params, dims, c)
    assert np.array_equal(got, ref)
    tgt = r.standard_normal(500)
    L, g, _, d_enc, _ = precision.grads_bf16(levels, bases, table, params, dims, c, tgt)
    y, a, z = mlp.forward(params, dims, encode.encode(levels, bases, c, table.astype(np.float64)))
    L0, gy = mlp.mse(y, tgt)
    g0, d0 = mlp.backward(params, dims, a, z, gy)
    assert L == L0 and np.array_equal(g, g0) and np.array_equal(d_enc, d0)


def test_grads_match_straight_through_autograd():
    """grads_bf16 against torch float64 autograd: each layer's value is the bf16-form pre-activation
    (bf16 inputs and weights, float32 bias), passed straight through, so autograd differentiates
    z = a W^T + b with the float32 master weights W and the activations a of the bf16 forward."""
    r = np.random.default_rng(5)
    levels = [[3, 3, 3, 2], [5, 4, 6, 3]]
    from oracle import schedule
    bases, rows = schedule.bases(levels)
    F = 2
    dims = [len(levels) * F, 16, 16, 1]
    table = (r.standard_normal((rows, F)) * 0.7).astype(np.float32)
    params = (r.standard_normal(mlp.n_params(dims)) * 0.4).astype(np.float32).astype(np.float64)
    c = r.random((300, 4)).astype(np.float32)
    tgt = r.standard_normal(300)
    L, g, _, d_enc, _ = precision.grads_bf16(levels, bases, table, params, dims, c, tgt)

    enc = torch.from_numpy(encode.encode(levels, bases, c, precision.bf16_round(table))).requires_grad_(True)
    bf = lambda t: t.detach().to(torch.bfloat16).to(torch.float64)   # noqa: E731
    leaves, x, o = [], enc, 0
    # (the encoding leaf's gradient is d(loss)/d(encoding): straight through the layer-1 rounding too)
    for k in range(len(dims) - 1):
        fi, fo = dims[k], dims[k + 1]
        W = torch.tensor(params[o:o + fo * fi].reshape(fo, fi), requires_grad=True)
        b = torch.tensor(params[o + fo * fi:o + fo * fi + fo], requires_grad=True)
        o += fo * fi + fo
        leaves += [W, b]
        lin = x @ W.T + b
        val = bf(x) @ bf(W).T + b.detach()
        z = lin + (val - lin).detach()
        x = torch.relu(z) if k < len(dims) - 2 else z
    loss = torch.mean((x[:, 0] - torch.from_numpy(tgt)) ** 2)
    loss.backward()
    g_ref = torch.cat([t.grad.reshape(-1) for t in leaves]).numpy()
    assert abs(L - loss.item()) <= 1e-14 * L
    assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-15)
    assert np.allclose(d_enc, enc.grad.numpy(), rtol=1e-12, atol=1e-15)
    # and the emulation's rounding matters here: the plain float64 gradient is measurably different
    y, a, z = mlp.forward(params, dims, encode.encode(levels, bases, c, table.astype(np.float64)))
    g_plain, _ = mlp.backward(params, dims, a, z, mlp.mse(y, tgt)[1])
    assert np.abs(g_plain - g).max() > 1e-6
