"""The host-side packing of fe2_batch_create, read back through the host-only
fe2_batch_layout (no GPU needed), against its documented invariants:

- parts per RVE follow the cluster-size rule: the smallest power of two
  whose parts hold the plain node state, doubled while the FP32 kernel's
  element table does not fit;
- the node permutation keeps each RVE's range, puts free nodes first part by
  part (degree order inside a part) and then fixed nodes part by part;
- RCB parts have equal sizes to within one node;
- every CSR row lists exactly the node's neighbours, in the caller's
  neighbour order, so each element appears twice, once from each end;
- (part, index) of every entry matches the permuted neighbour id.
"""
import numpy as np
import pytest

import rve_inputs as ri

SMEM_OPTIN = 232448       # GB300 opt-in shared memory per block
NODE_BYTES = 96           # FP32 kernel bytes per node without its element table


def _min_parts(n, target, smem_optin=SMEM_OPTIN):
    cap = smem_optin - 16384
    C = 1
    while C < 16 and (-(-n // C) > target or NODE_BYTES * (-(-n // C) + 64) > cap):
        C *= 2
    return C


def _check_parts(nets, target, L, smem_optin=SMEM_OPTIN):
    """At least the minimal cluster; more only where the minimal one leaves
    the FP32 kernel without its element table (checked through the plan with
    the part count forced one step lower)."""
    import paper_2305_07030_gb300 as m
    for p, net in enumerate(nets):
        C, C0 = int(L["parts"][p]), _min_parts(net.n_nodes, target, smem_optin)
        assert C >= C0 and C & (C - 1) == 0 and C <= 16, (p, C, C0)
        P = m.plan([net], smem_optin=smem_optin, nodes_per_cta=target)
        if C < 16:
            assert P["staged"][0, 1] == 1, (p, C)
        if C > C0:
            b = int(np.floor(np.log2(net.n_nodes)))
            m.tuning_set({b: (C // 2, 0)})
            try:
                half = m.plan([net], smem_optin=smem_optin, nodes_per_cta=target)
            finally:
                m.tuning_set(None)
            assert list(half["parts"]) == [C // 2]
            assert half["staged"][0, 1] == 0, (p, C)


def _check(nets, target, L):
    node_off, elem_off = L["node_off"], L["elem_off"]
    for p, net in enumerate(nets):
        base, n = int(node_off[p]), net.n_nodes
        C = int(L["parts"][p])
        adj = [[] for _ in range(n)]
        for a, b in net.elems:
            adj[a].append(b)
            adj[b].append(a)
        deg = np.array([len(x) for x in adj])
        free = (net.fixed == 0) & (deg > 0)
        nfree = int(free.sum())
        perm = L["perm"][base:base + n] - base
        assert sorted(perm.tolist()) == list(range(n))
        assert free[perm[:nfree]].all() and not free[perm[nfree:]].any()
        inv = np.empty(n, np.int64)
        inv[perm] = np.arange(n)
        pf, pg = L["part_off"][p, 0], L["part_off"][p, 1]
        assert pf[0] == 0 and pf[C] == nfree and (np.diff(pf[:C + 1]) >= 0).all()
        assert (pf[C:] == nfree).all()
        assert pg[0] == 0 and pg[C] == n - nfree and (pg[C:] == n - nfree).all()
        sizes = [(pf[r + 1] - pf[r]) + (pg[r + 1] - pg[r]) for r in range(C)]
        assert max(sizes) - min(sizes) <= 1, sizes
        owner, local = np.empty(n, np.int64), np.empty(n, np.int64)
        for r in range(C):
            fr = perm[pf[r]:pf[r + 1]]  # free nodes of part r, caller ids
            key = [(-deg[i], i) for i in fr]
            assert key == sorted(key), "free nodes of a part not in degree order"
            fx = perm[nfree + pg[r]:nfree + pg[r + 1]]
            assert list(fx) == sorted(fx), "fixed nodes of a part not in id order"
            owner[fr] = r
            local[fr] = np.arange(len(fr))
            owner[fx] = r
            local[fx] = len(fr) + np.arange(len(fx))
        rp = L["rowptr"][base + p:base + p + n + 1]
        csr0 = 2 * int(elem_off[p])
        assert rp[0] == 0 and rp[-1] == 2 * len(net.elems)
        for k in range(n):
            i = perm[k]
            cols = L["col"][csr0 + rp[k]:csr0 + rp[k + 1]]
            nb = perm[cols]  # back to caller ids
            assert list(nb) == sorted(adj[i]), (p, k)
            cp = L["col_part"][csr0 + rp[k]:csr0 + rp[k + 1]]
            assert list(cp >> 16) == list(owner[nb]) and list(cp & 0xFFFF) == list(local[nb])


def _nets(sizes, seed):
    rng = np.random.default_rng(seed)
    return [ri.random_network(int(n), rng) for n in sizes]


@pytest.mark.parametrize("target", [0, 256, 1024])
def test_uneven_batch(target):
    nets = _nets([37, 300, 777, 2100, 5000], seed=31)
    import paper_2305_07030_gb300 as m
    L = m.layout(nets, nodes_per_cta=target)
    _check(nets, target or 1024, L)
    _check_parts(nets, target or 1024, L)


def test_isolated_node_is_held_fixed():
    import paper_2305_07030_gb300 as m
    rng = np.random.default_rng(32)
    base = ri.random_network(80, rng)
    X = np.vstack([base.X, [[0.5, 0.5, 0.5]]])
    iso = ri.Network(X=X, elems=base.elems, EA=base.EA,
                     fixed=np.append(base.fixed, 0).astype(np.uint8))
    L = m.layout([iso])
    _check([iso], 1024, L)
    # the isolated node sits among the fixed nodes
    nfree = int(L["part_off"][0, 0, 1])
    assert 80 in L["perm"][nfree:].tolist()


def test_smem_bounds_the_part_size():
    """A small shared-memory budget forces more parts than the node target."""
    import paper_2305_07030_gb300 as m
    nets = _nets([3000], seed=33)
    small = 16384 + NODE_BYTES * (800 + 64)
    L = m.layout(nets, smem_optin=small, nodes_per_cta=4096)
    assert _min_parts(3000, 4096, small) == 4
    _check_parts(nets, 4096, L, smem_optin=small)


def test_tuned_part_count_is_used_and_bounded():
    """A tuned cluster size for a size bucket is used when feasible; one
    below the minimal cluster is ignored."""
    import paper_2305_07030_gb300 as m
    nets = _nets([5000, 700], seed=35)
    try:
        m.tuning_set({12: (16, 256)})       # 4096 <= n < 8192
        L = m.layout(nets)
        assert list(L["parts"]) == [16, int(m.layout(nets[1:])["parts"][0])]
        _check(nets, 1024, L)
        m.tuning_set({12: (2, 0)})          # below the minimal 8 parts: ignored
        assert int(m.layout(nets[:1])["parts"][0]) == 8
        with pytest.raises(m.FE2Error, match="power of two"):
            m.tuning_set({12: (3, 0)})
        with pytest.raises(m.FE2Error, match="multiples of 32"):
            m.tuning_set({12: (4, 100)})
    finally:
        m.tuning_set(None)
    assert m.tuning_get() == {}


def test_rejects_tiny_shared_memory():
    import paper_2305_07030_gb300 as m
    with pytest.raises(m.FE2Error, match="smem_optin"):
        m.layout(_nets([50], seed=34), smem_optin=4096)


def test_fp64_cluster_slot_tables():
    """The FP64 cluster kernel's element slots (fe2_batch_fp64_slots): per
    part one slot per element with an end among the part's free nodes, each
    once; every CSR entry of a free node points at the slot of its own
    element in its own part, with the orientation bit set exactly when the
    node is the element's second end in the caller's numbering; the slot's
    ends carry the (part << 16 | index) of col_part."""
    import paper_2305_07030_gb300 as m
    rng = np.random.default_rng(71)
    nets = [ri.random_network(int(n), rng) for n in (300, 1700, 4100)]
    L = m.layout(nets, smem_optin=SMEM_OPTIN)
    T = m.fp64_slots(nets, smem_optin=SMEM_OPTIN)
    slots, csr = T["slot"], T["csr_slot"]
    assert T["n_slots"] == len(slots) and T["slot0"][0] == 0
    for p, net in enumerate(nets):
        n0, e0 = int(L["node_off"][p]), int(L["elem_off"][p])
        C = int(L["parts"][p])
        pf = L["part_off"][p, 0]
        ps = T["part_slot"][p]
        base = int(T["slot0"][p])
        perm = L["perm"][n0:n0 + net.n_nodes] - n0          # permuted -> caller id
        rp = L["rowptr"][n0 + p:n0 + p + net.n_nodes + 1]
        csr0 = 2 * e0
        edge = {}
        for e, (a, b) in enumerate(net.elems):
            edge[(int(a), int(b))] = edge[(int(b), int(a))] = e
        for r in range(C):
            own = slots[base + ps[r]:base + ps[r + 1]]
            assert len(set(own[:, 0].tolist())) == len(own)  # each element once per part
            used = set()
            for k in range(pf[r], pf[r + 1]):                # the part's free nodes
                i = int(perm[k])
                for q in range(rp[k], rp[k + 1]):
                    w = int(csr[csr0 + q])
                    assert w >= 0
                    sl = own[w >> 1]
                    j = int(perm[L["col"][csr0 + q]])
                    e = edge[(i, j)]
                    assert sl[0] == e
                    a, b = (int(x) for x in net.elems[e])
                    assert (w & 1) == (1 if i == b else 0)
                    # the far end's (part, index) matches col_part of this entry
                    far = sl[2] if i == a else sl[1]
                    assert far == L["col_part"][csr0 + q]
                    used.add(w >> 1)
            assert used == set(range(len(own)))              # no slot unused
        for r in range(C, 16):
            assert ps[r + 1] == ps[C]
