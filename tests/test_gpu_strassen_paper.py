"""Sections "StrassenNaiv" and "StrassenWinograd" with the paper's own depth
rule (cutoff = 0: X = max{N, P, M}, k = floor(log2 X) - 4, Y = (floor(X/2^k) + 1)
2^k) at the sweep's sizes, through the C ABI against the CPU oracle's
recursion: exact on integer inputs, within 1e-14 normwise on uniform reals;
the depth-first split of the top levels gives the same bits as the
breadth-first plan; the whole recursion takes a few dozen launches."""
import os

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL = 1e-14
VARIANTS = [("strassen", "strassen_naiv"), ("strassen_winograd", "strassen_winograd")]


@pytest.fixture(scope="module")
def mm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1106_1347_gb300 import build

    build.build()
    import paper_1106_1347_gb300 as mm

    mm.lib()
    return mm


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t):
    return t.cpu().numpy()


@pytest.fixture
def breadth_cap():
    """Sets MM_STRASSEN_BREADTH_CAP for one test and restores it after."""
    old = os.environ.get("MM_STRASSEN_BREADTH_CAP")

    def set_cap(v):
        if v is None:
            os.environ.pop("MM_STRASSEN_BREADTH_CAP", None)
        else:
            os.environ["MM_STRASSEN_BREADTH_CAP"] = str(int(v))

    yield set_cap
    set_cap(None if old is None else int(old))


@pytest.mark.parametrize("gpu_name,orc_name", VARIANTS)
@pytest.mark.parametrize("n", [1024, 2047])
def test_paper_rule_sweep_sizes(mm, orc, gpu_name, orc_name, n):
    k, y = orc.strassen_paper_rule(n, n, n)
    assert k == 6 and y == (1088 if n == 1024 else 2048)
    ai = S.integers(n, n, S.stream_seed(1, 40))
    bi = S.integers(n, n, S.stream_seed(1, 41))
    assert np.array_equal(host(getattr(mm, gpu_name)(dev(ai), dev(bi), cutoff=0)), ai @ bi)
    a = S.uniform(n, n, S.stream_seed(1, 42))
    b = S.uniform(n, n, S.stream_seed(1, 43))
    got = host(getattr(mm, gpu_name)(dev(a), dev(b), cutoff=0))
    assert orc.rel_inf_error(got, getattr(orc, orc_name)(a, b), a, b) <= TOL


@pytest.mark.parametrize("gpu_name,orc_name", VARIANTS)
@pytest.mark.parametrize("shape", [(1000, 37, 513), (31, 700, 64), (513, 512, 511)])
def test_paper_rule_rectangular(mm, orc, gpu_name, orc_name, shape):
    ai = S.integers(shape[0], shape[1], S.stream_seed(1, 44))
    bi = S.integers(shape[1], shape[2], S.stream_seed(1, 45))
    assert np.array_equal(host(getattr(mm, gpu_name)(dev(ai), dev(bi), cutoff=0)), ai @ bi)
    a = S.uniform(shape[0], shape[1], S.stream_seed(1, 46))
    b = S.uniform(shape[1], shape[2], S.stream_seed(1, 47))
    got = host(getattr(mm, gpu_name)(dev(a), dev(b), cutoff=0))
    assert orc.rel_inf_error(got, getattr(orc, orc_name)(a, b), a, b) <= TOL


@pytest.mark.parametrize("gpu_name", ["strassen", "strassen_winograd"])
@pytest.mark.parametrize("shape,cutoff", [((200, 200, 200), 0), ((1024, 1024, 1024), 0), ((300, 257, 190), 80),
                                          ((1000, 600, 500), 300), ((256, 256, 256), 64)])
def test_depth_first_split_gives_the_same_bits(mm, breadth_cap, gpu_name, shape, cutoff):
    a = S.uniform(shape[0], shape[1], S.stream_seed(1, 48))
    b = S.uniform(shape[1], shape[2], S.stream_seed(1, 49))
    breadth_cap(None)
    whole = host(getattr(mm, gpu_name)(dev(a), dev(b), cutoff=cutoff))
    for cap in (1, 1 << 20):  # every level but the last depth-first; a few levels depth-first
        breadth_cap(cap)
        split = host(getattr(mm, gpu_name)(dev(a), dev(b), cutoff=cutoff))
        assert np.array_equal(split, whole), cap


def test_workspace_query_follows_the_cap(mm, breadth_cap):
    L = mm.lib()
    breadth_cap(None)
    whole = L.mm_strassen_workspace_bytes(1024, 1024, 1024, 0)
    breadth_cap(1)
    split = L.mm_strassen_workspace_bytes(1024, 1024, 1024, 0)
    assert 0 < split < whole


def test_paper_rule_is_a_few_launches(mm):
    a = dev(S.uniform(1024, 1024, S.stream_seed(1, 50)))
    b = dev(S.uniform(1024, 1024, S.stream_seed(1, 51)))
    mm.strassen(a, b, cutoff=0)
    with mm.profile() as prof:
        mm.strassen(a, b, cutoff=0)
    launches = sum(v[0] for v in prof.stats.values())
    assert launches <= 20, prof.stats  # depth 6: 3 expansion passes per side, 1 leaf pass, 3 combine passes
    assert "strassen_leaf_level" in prof.stats
