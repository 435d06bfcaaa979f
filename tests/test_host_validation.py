"""fe2_batch_create validates its inputs on the host before any device call,
so every rejection below is checked without a GPU: the call returns
FE2_EINVAL (1) with a message naming the problem, and never crashes."""
import ctypes as C

import numpy as np
import pytest

import rve_inputs as ri

FE2_EINVAL = 1


def _create(net, **over):
    """Call fe2_batch_create for one RVE; `over` replaces packed arrays."""
    import paper_2305_07030_gb300 as m
    a = {
        "node_off": np.array([0, net.n_nodes], np.int64),
        "X": np.ascontiguousarray(net.X, np.float64).reshape(-1),
        "elem_off": np.array([0, len(net.elems)], np.int64),
        "conn": np.ascontiguousarray(net.elems, np.int32).reshape(-1),
        "EA": np.ascontiguousarray(net.EA, np.float64),
        "fixed": np.ascontiguousarray(net.fixed, np.uint8),
        "V0": None,
        "damping": None,
    }
    a.update(over)
    h = C.c_void_p()
    p = lambda v: None if v is None else v.ctypes.data_as(C.c_void_p)  # noqa: E731
    rc = m._lib.fe2_batch_create(1, p(a["node_off"]), p(a["X"]), p(a["elem_off"]), p(a["conn"]),
                                 p(a["EA"]), p(a["fixed"]), p(a["V0"]), p(a["damping"]), None,
                                 C.byref(h))
    if rc == 0:  # a usable GPU: release what was made
        m._lib.fe2_batch_destroy(h)
    return rc, m.last_error()


@pytest.fixture(scope="module")
def net():
    return ri.random_network(40, np.random.default_rng(7))


def test_out_of_range_node(net):
    conn = np.ascontiguousarray(net.elems, np.int32).reshape(-1).copy()
    conn[5] = net.n_nodes
    rc, msg = _create(net, conn=conn)
    assert rc == FE2_EINVAL and "out of range" in msg


def test_negative_node(net):
    conn = np.ascontiguousarray(net.elems, np.int32).reshape(-1).copy()
    conn[0] = -1
    rc, msg = _create(net, conn=conn)
    assert rc == FE2_EINVAL and "out of range" in msg


def test_self_loop(net):
    conn = np.ascontiguousarray(net.elems, np.int32).reshape(-1).copy()
    conn[1] = conn[0]
    rc, msg = _create(net, conn=conn)
    assert rc == FE2_EINVAL and "itself" in msg


def test_repeated_element_either_orientation(net):
    e = np.ascontiguousarray(net.elems, np.int32)
    dup = np.vstack([e, e[3:4, ::-1]])  # the same element, reversed
    rc, msg = _create(net, conn=dup.reshape(-1).copy(),
                      elem_off=np.array([0, len(dup)], np.int64),
                      EA=np.append(net.EA, 1.0))
    assert rc == FE2_EINVAL and "repeats" in msg


@pytest.mark.parametrize("bad", [0.0, -1.0, np.inf, np.nan])
def test_bad_axial_stiffness(net, bad):
    EA = np.ascontiguousarray(net.EA, np.float64).copy()
    EA[2] = bad
    rc, msg = _create(net, EA=EA)
    assert rc == FE2_EINVAL and "EA" in msg


def test_zero_length_element(net):
    X = np.ascontiguousarray(net.X, np.float64).copy()
    a, b = net.elems[0]
    X[b] = X[a]
    rc, msg = _create(net, X=X.reshape(-1))
    assert rc == FE2_EINVAL and ("zero length" in msg or "repeats" in msg)


def test_non_finite_coordinate(net):
    X = np.ascontiguousarray(net.X, np.float64).copy()
    X[3, 1] = np.nan
    rc, msg = _create(net, X=X.reshape(-1))
    assert rc == FE2_EINVAL and "non-finite" in msg


@pytest.mark.parametrize("V0", [0.0, -2.0, np.nan])
def test_bad_reference_volume(net, V0):
    rc, msg = _create(net, V0=np.array([V0]))
    assert rc == FE2_EINVAL and "V0" in msg


@pytest.mark.parametrize("c", [-0.1, np.inf])
def test_bad_damping(net, c):
    rc, msg = _create(net, damping=np.array([c]))
    assert rc == FE2_EINVAL and "damping" in msg


def test_offsets(net):
    rc, msg = _create(net, node_off=np.array([1, net.n_nodes], np.int64))
    assert rc == FE2_EINVAL and "start at 0" in msg
    rc, msg = _create(net, node_off=np.array([0, 0], np.int64))
    assert rc == FE2_EINVAL and "no nodes" in msg


def test_valid_input_passes_validation(net):
    """A valid RVE gets past validation: OK on a GB300, otherwise a device
    error (never FE2_EINVAL), reported through the status."""
    rc, msg = _create(net)
    assert rc != FE2_EINVAL, msg
    if rc != 0:
        assert msg
