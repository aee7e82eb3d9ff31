"""The allocation-free entry point ttns_rho_from_root_noalloc against the regular
ttns_reduced_density_matrix, through the C ABI, on two calls in a row.

This is for callers that cannot call cudaMalloc (for example code running inside
another framework's locked memory pool): the caller passes its own device buffers
and the library uses a fixed scratch array instead of allocating.  Kept in its own
file so that it is collected last.
"""
import numpy as np
import pytest

from paper_1710_01362_gb300 import build, ttns
from paper_1710_01362_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_noalloc_density_matches_the_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    p = W.sf_small(seed=7)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    n_el = p.n_el
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):          # two calls in a row, on different states
        g.step(p.dt, 3)
        root = g.node(0)           # host copy through the public API
        rows = root.size // n_el
        d_root = torch.from_numpy(np.ascontiguousarray(root).view(np.float64).reshape(-1)).cuda()
        d_rho = torch.full((2 * n_el * n_el,), float("nan"), dtype=torch.float64, device="cuda")
        ttns.rho_from_root_noalloc(d_root.data_ptr(), rows, n_el, d_rho.data_ptr(), stream)
        torch.cuda.synchronize()
        got = d_rho.cpu().numpy().view(np.complex128).reshape(n_el, n_el)
        ref = g.rho()
        assert np.abs(got - ref).max() < 1e-12, f"call {call}"
    with pytest.raises(ttns.TTNSError) as e:
        ttns.rho_from_root_noalloc(d_root.data_ptr(), rows, 17, d_rho.data_ptr(), stream)
    assert e.value.code == 1
    g.close()


def test_noalloc_density_at_the_scratch_limits():
    # rows = 20000, n_el = 16: 256 blocks of 16 x 16 partials, the whole fixed scratch array,
    # against a plain einsum on the host; then a size at the 2^24 element limit is rejected
    # before anything is launched
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    rng = np.random.default_rng(5)
    rows, n_el = 20000, 16
    A = (rng.standard_normal((rows, n_el)) + 1j * rng.standard_normal((rows, n_el))) / np.sqrt(rows)
    ref = np.einsum("rs,rt->st", A, A.conj())
    stream = torch.cuda.current_stream().cuda_stream
    d_root = torch.from_numpy(np.ascontiguousarray(A).view(np.float64).reshape(-1)).cuda()
    for call in range(2):
        d_rho = torch.full((2 * n_el * n_el,), float("nan"), dtype=torch.float64, device="cuda")
        ttns.rho_from_root_noalloc(d_root.data_ptr(), rows, n_el, d_rho.data_ptr(), stream)
        torch.cuda.synchronize()
        got = d_rho.cpu().numpy().view(np.complex128).reshape(n_el, n_el)
        assert np.abs(got - ref).max() < 1e-12, f"call {call}"
    with pytest.raises(ttns.TTNSError) as e:
        ttns.rho_from_root_noalloc(d_root.data_ptr(), (1 << 24) // n_el, n_el, d_rho.data_ptr(), stream)
    assert e.value.code == 1
