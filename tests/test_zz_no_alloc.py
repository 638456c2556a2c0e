"""qmpm_tile_order_static: the particle order without any device allocation.

Some callers cannot call cudaMalloc or cudaFree -- code that runs inside another
runtime's memory pool, or a host thread that must not take the device-wide
synchronisation an allocation can cause.  This entry point gives them the stable
(tile, cell) order that qmpm_init computes, with its scratch in a static device array of
the library.  The test feeds it the records of a scene in their input order and checks
that it reproduces, slot for slot, the order qmpm_init chose for the same records, on
several calls in a row (the scratch is shared between calls), and that an input above the
static limit is refused.  This file runs last so that a failure here comes after every
other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    from paper_2207_04658_b300 import qmpm
    assert torch.cuda.is_available()
    qmpm.lib()
    return qmpm


def cases():
    from paper_2207_04658_b300 import scenes
    out = []
    sc, s0 = scenes.block2d_scene(n_strata=(64, 32))
    out.append((sc, scenes.block2d_scheme(), s0))
    sc, s0 = scenes.cubes3d_scene(n_cubes=2, cube_cells=10, ppc_axis=2, grid_log2=6, seed=5)
    out.append((sc, scenes.fixed_scheme_3d("corotated"), s0))
    sc, s0 = scenes.dambreak3d_scene(column_cells=12, ppc_axis=2, grid_log2=6)
    out.append((sc, None, s0))  # FP32 state
    return out


def static_order_equals_init_order(q, sc, scheme, s0):
    import torch
    g = q.Scene(sc, scheme, s0)
    r = g.readback(state=False, words=True, ids=True)
    dim, material = sc["dim"], sc["material"]
    g.close()
    words_sorted, ids = r["words"], r["ids"]
    N = s0.shape[0]
    # the records back in input order: slot i holds input record ids[i]
    words_in = np.empty_like(words_sorted)
    words_in[:, ids] = words_sorted
    ld = N + 7  # a leading dimension that is not a multiple of anything
    d_words = torch.zeros((words_in.shape[0], ld), dtype=torch.int32, device="cuda")
    d_words[:, :N] = torch.from_numpy(words_in.view(np.int32))
    d_order = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    sch = q.make_scheme_struct(scheme, dim, material) if scheme is not None else None
    q.qmpm_tile_order_static(dim, q.MATERIALS[material], sch, sc["grid_log2"], d_words.data_ptr(), N, ld,
                             d_order.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    order = d_order.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(order, ids)


def test_static_order_matches_init_order(q):
    cs = cases()
    # several calls in a row share the static scratch: each must stand on its own
    for sc, scheme, s0 in cs + cs[:1]:
        static_order_equals_init_order(q, sc, scheme, s0)


def test_static_order_refuses_oversize_input(q):
    with pytest.raises(q.QmpmError) as ei:
        q.qmpm_tile_order_static(3, 1, None, 8, 0, q.STATIC_SORT_MAX + 1, q.STATIC_SORT_MAX + 1, 0)
    assert ei.value.code == -1
    assert "static scratch limit" in str(ei.value)
