"""Failure paths and checkpoints of the C ABI on the GPU.

Every failure here is made on the host: a checkpoint file with a NaN written into
it, a Krylov tolerance no space can reach, a launch with a cluster shape the
kernel's own launch check refuses.  None faults, traps or hangs the GPU: the
kernel reports each one through its status word and returns.
"""
import struct

import numpy as np
import pytest

from paper_1710_01362_gb300 import build, ttns
from paper_1710_01362_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_checkpoint_with_a_nan_tensor_reports_nonfinite(tmp_path):
    p = W.sf_small(seed=7)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    g.step(p.dt, 2)
    first = g.node(0).reshape(-1)[0]
    path = str(tmp_path / "nan.ck")
    g.save(path)
    g.close()
    data = bytearray(open(path, "rb").read())
    key = struct.pack("<dd", first.real, first.imag)
    at = data.find(key)
    assert at > 0 and data.find(key, at + 1) < 0, "root element not unique in the file"
    data[at:at + 8] = struct.pack("<d", float("nan"))
    open(path, "wb").write(bytes(data))
    h = ttns.Tree.load(path, p, precision=ttns.TTNS_FP64)  # contents are not validated on load
    h.step(p.dt, 1)
    with pytest.raises(ttns.TTNSError) as e:
        h.sync()
    assert e.value.code == 6, str(e.value)
    h.close()


def test_unreachable_krylov_tolerance_reports_not_converged():
    # no Krylov space of dimension 3 reaches 1e-300: every space takes s / 2^30 and the
    # 64 spaces of one exponential do not cover the half step
    p = W.spin_boson(L=4, d=4, D=4, n_steps=1)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64, krylov_mmax=3, krylov_tol=1e-300)
    g.step(p.dt, 1)
    with pytest.raises(ttns.TTNSError) as e:
        g.sync()
    assert e.value.code == 4, str(e.value)
    assert g.counters()["not_converged"] >= 1
    g.close()


@pytest.mark.parametrize("prec", [ttns.TTNS_FP64, ttns.TTNS_MIXED])
def test_load_builds_the_tree_from_the_file_alone(tmp_path, prec):
    p = W.sf_small(seed=7)
    a = ttns.Tree(p, precision=prec, record=True, max_record=16)
    a.step(p.dt, 5)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(p.dt, 5)
    b = ttns.Tree.load(path, p, precision=prec)
    b.step(p.dt, 5)
    assert np.array_equal(a.rho(), b.rho())
    assert np.array_equal(a.trajectory(), b.trajectory())
    assert np.array_equal(a.occupations(), b.occupations())
    a.close()
    b.close()
    with pytest.raises(ttns.TTNSError) as e:
        ttns.Tree.load(str(tmp_path / "missing.bin"), p)
    assert e.value.code == 7


def test_refused_launch_is_repeated_as_a_plain_cluster_launch():
    # launch_flags bit 1: the first step launch gets clusters of one CTA; the kernel's
    # launch check refuses it before any work, and the library repeats it with the planned
    # clusters (no cooperative attribute).  The result equals an ordinary run bit for bit.
    p = W.sf_small(seed=7)
    r = []
    fallbacks = []
    for flags in (0, 2):
        g = ttns.Tree(p, precision=ttns.TTNS_MIXED, grid_threshold=64, launch_flags=flags)
        g.step(p.dt, 3)
        r.append(g.rho())
        fallbacks.append(g.counters()["launch_fallbacks"])
        g.close()
    assert fallbacks == [0, 1]
    assert np.array_equal(r[0], r[1])


def test_refused_step_launch_is_repeated_with_every_pending_step():
    # two step launches are pending when the refusal is seen: both are repeated, in order
    p = W.sf_small(seed=7)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    g.step(p.dt, 2)
    g.step(p.dt, 1)
    ref = g.rho()
    g.close()
    h = ttns.Tree(p, precision=ttns.TTNS_FP64, launch_flags=2)
    h.step(p.dt, 2)
    h.step(p.dt, 1)
    assert np.array_equal(h.rho(), ref)
    h.close()
