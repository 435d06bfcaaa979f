"""The mixed solver's launch plan, read back through the host-only
fe2_batch_plan (no GPU needed)."""
import numpy as np
import pytest

import rve_inputs as ri

SMEM_OPTIN = 232448  # GB300 opt-in shared memory per block


def test_benchmark_workload_runs_the_staged_kernels():
    """64 RVEs of 5000 nodes: one class of 8-CTA clusters whose element
    tables fit in shared memory for both kernels (the fast paths), 512
    threads per CTA. A change that grows the per-node or per-element shared
    memory past the budget would silently move this workload to the
    re-reading fallback; this test catches it."""
    import paper_2305_07030_gb300 as m
    w = ri.equal_rves(64, 5000)
    P = m.plan(w.nets, smem_optin=SMEM_OPTIN)
    assert P["n_classes"] == 1 and list(P["parts"]) == [8] and list(P["rves"]) == [64]
    assert P["staged"].tolist() == [[1, 1]]
    assert P["block"].tolist() == [[512, 512]]
    assert (P["smem"] <= SMEM_OPTIN - 16384).all()


@pytest.mark.parametrize("target", [0, 256])
def test_plan_is_consistent_with_the_layout(target):
    import paper_2305_07030_gb300 as m
    rng = np.random.default_rng(41)
    nets = [ri.random_network(int(n), rng) for n in (37, 300, 777, 2100, 5000, 9000, 120)]
    P = m.plan(nets, smem_optin=SMEM_OPTIN, nodes_per_cta=target)
    L = m.layout(nets, smem_optin=SMEM_OPTIN, nodes_per_cta=target)
    k = P["n_classes"]
    assert sum(P["rves"]) == len(nets)
    # every RVE in a class of its own cluster size; a class is one cluster
    # size and one choice of element tables for each kernel
    for p in range(len(nets)):
        assert P["parts"][P["rve_class"][p]] == L["parts"][p]
    keys = [(int(P["parts"][c]), *map(int, P["staged"][c])) for c in range(k)]
    for c in range(k):
        for p in np.nonzero(P["rve_class"] == c)[0]:
            alone = m.plan([nets[p]], smem_optin=SMEM_OPTIN, nodes_per_cta=target)
            assert (int(alone["parts"][0]), *map(int, alone["staged"][0])) == keys[c]
            assert alone["block"].tolist() == [P["block"][c].tolist()]
    assert np.bincount(P["rve_class"], minlength=k).tolist() == P["rves"].tolist()
    # every launch fits the shared-memory budget; the lead kernel without its
    # table runs 256 threads per CTA, everything else 512
    assert (P["smem"] <= SMEM_OPTIN - 16384).all()
    for c in range(k):
        lead_staged, fp32_staged = P["staged"][c]
        assert P["block"][c, 0] == (512 if lead_staged else 256)
        assert P["block"][c, 1] == 512


def test_small_shared_memory_needs_more_parts():
    """With less shared memory the same RVEs need at least as many parts;
    a plan never exceeds the budget."""
    import paper_2305_07030_gb300 as m
    rng = np.random.default_rng(42)
    nets = [ri.random_network(int(n), rng) for n in (800, 1600)]
    big = m.plan(nets, smem_optin=SMEM_OPTIN)
    small_optin = 120 * 1000
    small = m.plan(nets, smem_optin=small_optin)
    assert (small["smem"] <= small_optin - 16384).all()
    for p in range(len(nets)):
        assert small["parts"][small["rve_class"][p]] >= big["parts"][big["rve_class"][p]]


def test_mixed_path_size_limit():
    """The mixed solver holds each part's node state in shared memory (96 B
    per node without the element table), so on a GB300 an RVE fits in 16
    parts of at most 2,250 nodes; the bisection leaves parts within one node
    of each other, so 36,000 nodes fit and 36,017 do not. The header states
    the guaranteed 34,976 (parts of 2,186 with slack for the bisection)."""
    import paper_2305_07030_gb300 as m
    budget = SMEM_OPTIN - 16384
    assert budget // 96 == 2250
    for n, fits in ((34_976, True), (36_000, True), (36_017, False)):
        P = m.plan([ri.random_network(n, np.random.default_rng(43))], smem_optin=SMEM_OPTIN)
        assert list(P["parts"]) == [16]
        assert bool((P["smem"] <= budget).all()) == fits, (n, P["smem"].tolist())


def test_plan_of_an_uneven_batch_with_many_classes():
    """The 64 size-stratified RVEs of the 4096 x log-U(500, 20k) workload
    split into more than eight launch classes (cluster size and staging per
    RVE); every RVE is in exactly one class, every class fits, and an RVE's
    class key does not depend on the batch it is in."""
    import paper_2305_07030_gb300 as m
    idx = ri.stratified_idx(ri.uneven_sizes(4096, 500, 20000, 4), 64)
    w = ri.uneven_subset(4096, 500, 20000, 4, idx)
    P = m.plan(w.nets, smem_optin=SMEM_OPTIN)
    k = P["n_classes"]
    assert k > 8 and len(P["parts"]) == k
    assert int(P["rves"].sum()) == 64
    assert np.array_equal(np.bincount(P["rve_class"], minlength=k), P["rves"])
    assert (P["smem"] <= SMEM_OPTIN - 16384).all()
    for p in (0, 31, 63):
        alone = m.plan([w.nets[p]], smem_optin=SMEM_OPTIN)
        c = P["rve_class"][p]
        assert (int(alone["parts"][0]), *map(int, alone["staged"][0])) == \
            (int(P["parts"][c]), *map(int, P["staged"][c]))
