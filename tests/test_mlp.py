"""Warm-start network: the FP64 oracle MLP pinned by finite differences (CPU);
the CUDA forward/backward checked against it, training and bfloat16
inference, and the warm start's gain over theta = 0 on held-out targets (GPU)."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def _params(d, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(len(d) - 1):
        out.append(rng.normal(0, np.sqrt(2.0 / (d[k] + d[k + 1])), size=d[k] * d[k + 1]))
        out.append(rng.normal(0, 0.1, size=d[k + 1]))
    return np.concatenate(out)


def test_oracle_mlp_gradient_by_finite_differences():
    d = mo.widths(5, 7, 3, 4)
    p = _params(d, 0)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(6, 5))
    T = rng.normal(size=(6, 4))
    loss, g = mo.loss_and_grad(p, d, X, T)
    h = 1e-6
    idx = rng.choice(p.size, 40, replace=False)
    for i in idx:
        e = np.zeros(p.size)
        e[i] = h
        fd = (mo.loss_and_grad(p + e, d, X, T)[0] - mo.loss_and_grad(p - e, d, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i]))


def test_oracle_gelu_closed_values():
    # x Phi(x): Phi(0) = 1/2, Phi(1) = 0.841344746068543, gelu'(0) = 1/2
    assert mo.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mo.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-15
    assert abs(mo.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


@pytest.mark.gpu
def test_gpu_mlp_gradient_matches_oracle():
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build
    build.build()
    n_in, hid, nh, n_out = 64, 256, 3, 64
    d = mo.widths(n_in, hid, nh, n_out)
    p = _params(d, 2).astype(np.float32)
    rng = np.random.default_rng(3)
    X = rng.normal(size=(37, n_in)).astype(np.float32)      # ragged batch
    T = rng.normal(size=(37, n_out)).astype(np.float32)
    m = q.MLP(n_in, hid, nh, n_out, p, max_batch=64)
    loss, g = m.gradient(X, T)
    loss_o, g_o = mo.loss_and_grad(p.astype(float), d, X.astype(float), T.astype(float))
    assert abs(loss - loss_o) <= 1e-5 * loss_o
    assert np.linalg.norm(g - g_o) <= 1e-5 * np.linalg.norm(g_o)
    y32 = m.predict(X, bf16=False)
    y_o, _ = mo.forward(p.astype(float), d, X.astype(float))
    assert np.linalg.norm(y32 - y_o) <= 1e-5 * np.linalg.norm(y_o)
    y16 = m.predict(X, bf16=True)           # bfloat16 weights and activations: ~2-3 significant digits
    assert np.linalg.norm(y16 - y_o) <= 2e-2 * np.linalg.norm(y_o)
    m.close()


def _bf16(x):
    """Round binary32 values to bfloat16 (nearest, ties to even), kept as binary32."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def _bf16_forward(params, d, X):
    """The network with every layer's weights and input activations rounded
    to bfloat16, products and sums in binary64, bias and GELU in binary64."""
    layers = mo.unpack(params, d)
    h = X.astype(np.float32)
    for k, (W, b) in enumerate(layers):
        z = _bf16(h).astype(float) @ _bf16(W.astype(np.float32)).astype(float) + b.astype(np.float32)
        h = (mo.gelu(z) if k < len(layers) - 1 else z).astype(np.float32)
    return h.astype(float)


def test_bf16_rounding_helper():
    x = np.array([1.0, 1.00390625, 1.001953125, 1.005859375, -3.0e-3, 0.0], dtype=np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even (1); 1 + 3 * 2^-9 rounds up
    np.testing.assert_array_equal(_bf16(x)[:4], np.array([1.0, 1.0, 1.0, 1.0078125], dtype=np.float32))
    assert abs(_bf16(x)[4] + 3.0e-3) <= 3.0e-3 * 2.0 ** -8 and _bf16(x)[5] == 0.0


@pytest.mark.gpu
@pytest.mark.parametrize("shape,batch", [((64, 256, 3, 64), 37), ((64, 256, 3, 64), 200), ((8, 64, 2, 4), 45)])
def test_gpu_mlp_bf16_tensor_core_inference(shape, batch):
    """bfloat16 inference on the tensor cores against the same rounding done
    on the host with binary64 sums (only the binary32 accumulation order
    differs), and against the unrounded binary64 network (the bfloat16
    error itself)."""
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build
    build.build()
    n_in, hid, nh, n_out = shape
    d = mo.widths(n_in, hid, nh, n_out)
    p = _params(d, 7).astype(np.float32)
    X = np.random.default_rng(8).normal(size=(batch, n_in)).astype(np.float32)
    m = q.MLP(n_in, hid, nh, n_out, p, max_batch=256)
    y16 = m.predict(X, bf16=True).astype(float)
    m.close()
    y_r = _bf16_forward(p, d, X)
    y_o, _ = mo.forward(p.astype(float), d, X.astype(float))
    assert np.linalg.norm(y16 - y_r) <= 2e-4 * np.linalg.norm(y_r)
    assert np.abs(y16 - y_r).max() <= 2e-3 * np.abs(y_r).max()
    assert np.linalg.norm(y16 - y_o) <= 2e-2 * np.linalg.norm(y_o)


@pytest.mark.gpu
def test_gpu_mlp_training_fits_a_smooth_map():
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, warmstart
    build.build()
    rng = np.random.default_rng(4)
    X = rng.normal(size=(512, 8)).astype(np.float32)
    A = rng.normal(size=(8, 4))
    T = np.tanh(X @ A).astype(np.float32)
    m = q.MLP(8, 64, 2, 4, warmstart.init_params(8, 64, 2, 4, 5), max_batch=128)
    m.set_dataset(X, T)
    perms = np.stack([rng.permutation(512) for _ in range(150)])
    losses = m.train(perms, 64, 3e-3)
    assert losses[-1] < 0.05 * losses[0]
    m.close()


@pytest.mark.gpu
def test_gpu_warm_start_reduces_trust_region_iterations():
    """Trained on theta* from the library's own trust region, the network's
    theta0 needs fewer iterations than theta = 0 on held-out targets."""
    from paper_2505_00529_gb300 import build, inputs, warmstart
    import paper_2505_00529_gb300 as q
    build.build()
    prob = inputs.small_problem(N=6, K=8, J=200, seed=31, dt=0.05, basis="sine_cosine")
    train = inputs.random_targets(101, 6, 192)
    test = inputs.random_targets(202, 6, 24)
    r = warmstart.compare(prob, train, test, precision=q.QOC_FP64, workers=4, epochs=300, batch=64,
                          lr=2e-3, gtol=1e-7, xtol=1e-12, max_iter=200)
    assert r["converged_mlp"] >= r["converged_zero"] - 1e-9
    assert r["iters_mlp_mean"] < r["iters_zero_mean"], r


def test_newton_decrement():
    """g^T H^-1 g for a positive definite H (against a direct solve), +inf
    for an indefinite or singular one."""
    from paper_2505_00529_gb300 import warmstart
    rng = np.random.default_rng(3)
    A = rng.normal(size=(6, 6))
    H = A @ A.T + 0.5 * np.eye(6)
    g = rng.normal(size=6)
    assert np.isclose(warmstart.newton_decrement(g, H), g @ np.linalg.solve(H, g), rtol=1e-12)
    Hi = H - 10.0 * np.eye(6) * np.abs(np.linalg.eigvalsh(H)).max()
    assert warmstart.newton_decrement(g, Hi) == np.inf
    assert warmstart.newton_decrement(g, np.zeros((6, 6))) == np.inf
