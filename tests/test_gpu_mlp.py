"""The surrogate network's kernels (tensor-core layer products with fused epilogues,
backpropagation, Adam) against the FP64 CPU oracle of the same network (oracle/mlp.py,
pinned by finite differences), through the C ABI; and a small end-to-end surrogate run
whose fallback rows are the TTNS results themselves.

Tolerances: the 3xTF32 products are FP32-level (relative error ~1e-6 of the operand
scale, summed in round-to-nearest), so gradients agree with FP64 to 1e-4 of their own
scale; one BF16 product keeps 8 bits per operand, so the inference forward agrees to
2e-2 of the output scale.
"""
import numpy as np
import pytest

from paper_1710_01362_gb300 import build, ttns
from oracle import mlp as OM

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _gemm(kind, A, B, transA, transB, epi=0, aux=None):
    # C = op(A) op(B) with the stored layouts the transposes describe
    Ad = torch.tensor(A, dtype=torch.float32, device="cuda").contiguous()
    Bd = torch.tensor(B, dtype=torch.float32, device="cuda").contiguous()
    M = A.shape[1] if transA else A.shape[0]
    K = A.shape[0] if transA else A.shape[1]
    N = B.shape[0] if transB else B.shape[1]
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    auxd = None if aux is None else torch.tensor(aux, dtype=torch.float32, device="cuda").contiguous()
    code = ttns.lib().ttns_mlp_gemm(kind, M, N, K, Ad.data_ptr(), A.shape[1], transA, Bd.data_ptr(), B.shape[1],
                                    transB, C.data_ptr(), N, epi, None if auxd is None else auxd.data_ptr(), None)
    assert code == 0, ttns.lib().ttns_last_error()
    torch.cuda.synchronize()
    return C.double().cpu().numpy()


@pytest.mark.parametrize("kind,tol", [(1, 2e-6), (3, 2e-2)])
@pytest.mark.parametrize("M,N,K", [(256, 256, 30), (130, 1000, 256), (7, 9, 300), (256, 64, 256)])
def test_layer_product_all_layouts_and_epilogues(kind, tol, M, N, K):
    rng = np.random.default_rng(M + N + K + kind)
    A = rng.standard_normal((M, K)) / np.sqrt(K)
    B = rng.standard_normal((K, N))
    bias = rng.standard_normal(N)
    H = np.tanh(rng.standard_normal((M, N)))
    ref = A @ B
    scale = np.abs(A) @ np.abs(B)
    for ta, tb in ((0, 0), (1, 0), (0, 1), (1, 1)):
        Ast = A.T.copy() if ta else A
        Bst = B.T.copy() if tb else B
        C = _gemm(kind, Ast, Bst, ta, tb)
        assert (np.abs(C - ref) / scale).max() < tol, (ta, tb)
    C = _gemm(kind, A, B, 0, 0, 1, bias)
    assert (np.abs(C - (ref + bias)) / (scale + np.abs(bias))).max() < tol
    C = _gemm(kind, A, B, 0, 0, 2, bias)
    assert np.abs(C - np.tanh(ref + bias)).max() < 2 * tol * (scale + np.abs(bias)).max()
    C = _gemm(kind, A, B, 0, 0, 3, H)
    assert (np.abs(C - ref * (1 - H ** 2)) / scale).max() < tol


def _net_and_batch(widths, B, seed):
    from paper_1710_01362_gb300.surrogate import Net
    rng = np.random.default_rng(seed)
    params = OM.init_params(widths, seed)
    params = [(Wl, rng.normal(scale=0.1, size=bl.shape)) for Wl, bl in params]
    x = rng.standard_normal((B, widths[0]))
    t = rng.uniform(0, 1, size=(B, widths[-1]))
    net = Net(widths, seed=0)
    net.set_params(params)
    return net, params, x, t


def test_gradients_match_the_fp64_oracle():
    widths = [30, 64, 48, 40]
    net, params, x, t = _net_and_batch(widths, 96, 5)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    y, hs = net.forward(xd)
    grads = net.backward(hs, y, td)
    torch.cuda.synchronize()
    ref = OM.backward(params, x, t)
    y_ref, _ = OM.forward(params, x)
    assert np.abs(y.double().cpu().numpy() - y_ref).max() < 1e-4 * np.abs(y_ref).max()
    for l, ((dW, db), (rW, rb)) in enumerate(zip(grads, ref)):
        gW = dW.double().cpu().numpy()
        gb = db.double().cpu().numpy()
        assert np.abs(gW - rW).max() <= 1e-4 * np.abs(rW).max(), l
        assert np.abs(gb - rb).max() <= 1e-4 * np.abs(rb).max(), l


def test_adam_step_matches_the_oracle():
    widths = [30, 16, 12]
    net, params, x, t = _net_and_batch(widths, 32, 8)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    opt = OM.Adam(params, lr=1e-2)
    p_ref = params
    for _ in range(3):
        y, hs = net.forward(xd)
        net.adam(net.backward(hs, y, td), 1e-2)
        p_ref = opt.step(p_ref, OM.backward(p_ref, x, t))
    torch.cuda.synchronize()
    for l in range(len(widths) - 1):
        assert np.abs(net.W[l].double().cpu().numpy() - p_ref[l][0]).max() < 1e-4
        assert np.abs(net.b[l].double().cpu().numpy() - p_ref[l][1]).max() < 1e-4


def test_bf16_inference_against_fp64_forward():
    widths = [30, 256, 256, 256, 1000]
    net, params, x, t = _net_and_batch(widths, 200, 9)
    y, _ = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda"), kind=3)
    torch.cuda.synchronize()
    y_ref, _ = OM.forward(params, x)
    assert np.abs(y.double().cpu().numpy() - y_ref).max() < 2e-2 * np.abs(y_ref).max()


def test_small_surrogate_trains_and_falls_back_to_the_sweep():
    from paper_1710_01362_gb300 import surrogate as S
    n_points = 20
    kw = dict(n_points=n_points, L=2, d=3, D=3, dt=1.0)
    X, Y, _ = S.generate(range(600), **kw)
    assert np.allclose(Y.reshape(len(Y), n_points, 5).sum(axis=2), 1.0, atol=1e-4)  # populations sum to one
    sur = S.Surrogate(n_points=n_points, seed=3)
    sur.fit(X[:500], Y[:500], X[500:550], Y[500:550], epochs=30, batch=100, lr=3e-3, lr_final=1e-4)
    X_test, Y_test = X[550:], Y[550:]
    calls = []

    def fallback(rows):
        calls.append(rows)
        return Y_test[rows]             # the TTNS runs of those parameter sets

    Yp, perr, back = sur.predict(X_test, threshold=1e-3, fallback=fallback)
    err = np.abs(Yp - Y_test).max(axis=1)
    assert np.all(err[back] == 0.0)                     # fallback rows are the sweep's results
    baseline = np.abs(Y_test - Y[:500].mean(axis=0)).max(axis=1)
    assert np.median(err[~back] if (~back).any() else err) < np.median(baseline)  # it learned something
    assert len(calls) == (1 if back.any() else 0)
