"""The ablation runs (bench.py --ablations) on small inputs: the shapes of their results,
degrees within the cap, and the expected direction of the alpha study (a much wider
angle keeps far fewer edges)."""
import pytest

from paper_1907_06146_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ssg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06146_gb300 import build_ext, ssg as S
    build_ext.build()
    S.lib()
    return S


def test_alpha_sweep(ssg):
    from paper_1907_06146_gb300 import ablations
    w = synth.small(n=6000, nq=300)
    r = ablations.alpha_sweep(ssg, w, n=6000, nq=300, alphas=(30.0, 45.0, 60.0, 80.0))
    pts = {p["alpha"]: p for p in r["points"]}
    # at 30 degrees every reached node is full before the graph is connected (R = 32 on
    # 32-d data); the oracle stops there too, and the sweep records it
    assert "error" in pts[30.0] and "free slot" in pts[30.0]["error"]
    ok = [p for p in r["points"] if "error" not in p]
    assert pts[45.0]["avg_out_degree"] > pts[80.0]["avg_out_degree"]
    assert all(p["max_out_degree"] <= w.R for p in ok)
    # recall at the largest L_search tried, or the L_search that reached 0.95 and its QPS
    assert all(0.0 <= p["recall"] <= 1.0 for p in ok)
    assert all(p["qps"] is None or p["qps"] > 0 for p in ok)


def test_exact_vs_nssg_counts(ssg):
    from paper_1907_06146_gb300 import ablations
    r = ablations.exact_vs_nssg(ssg, synth, n=400, d=16)
    assert 0 < r["shared"] <= min(r["exact_edges"], r["nssg_edges"])
    assert 0.0 < r["exact_covered"] <= 1.0 and 0.0 < r["nssg_in_exact"] <= 1.0


def test_pool_variant_shapes(ssg):
    from paper_1907_06146_gb300 import ablations
    w = synth.sift_like(n=6000, nq=300, n_clusters=40)
    r = ablations.pool_variant(ssg, w, n=6000, nq=300)
    v = r["variants"]
    assert set(v) == {"as_printed", "own_row_first"}
    for p in v.values():
        assert 0 < p["avg_out_degree"] <= w.R and 0.0 <= p["recall"] <= 1.0
