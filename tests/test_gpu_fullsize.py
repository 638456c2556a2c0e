"""One step at the full sizes, in the launch configuration the benchmark times, against the
oracle over every particle (its threaded build, so that a full-size FP64 step takes
seconds on the host cores): the 3D elastic cubes (8,192,000 particles, 256^3, the cached
second-order scheme at eps = 0.01) and the 3D weakly compressible dam break (2^27 =
134,217,728 particles, 512^3, dithered and not).  Bars: the initial encode and the tile
order are bit-exact (same slots, same ids); after one step every stored value is within two
quanta of the oracle's (a rounding difference that crosses a dither threshold), and the
particles' mass is conserved by the grid (P2G of a known state).  Both with the library's
step kernel and with the kernel compiled for the scheme (QMPM_FLAG_SPECIALIZE)."""
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


def quanta(oracle, sc, sch):
    names = ["x", "v", "C", "J" if sc["material"] == "fluid" else "F"]
    return np.array([2.0 ** -sch[names[h]]["frac"] for h in oracle.comp_fields(sc["dim"], sc["material"])])


def one_step_parity(q, oracle, sc, s0, sch, block=1 << 24, spec=False):
    """Returns (largest difference in quanta, fraction of values that differ).  spec: step
    with the kernel compiled for the scheme (QMPM_FLAG_SPECIALIZE)."""
    g = q.Scene(sc, sch, s0, specialize=spec)
    assert q.qmpm_step_kernel_info(g.h)["specialized"] == spec
    o = oracle.QuantRollout(sc, sch, s0, threaded=True)
    w0 = g.readback(state=False, words=True, ids=True)
    assert np.array_equal(w0["ids"], o.ids)
    assert np.array_equal(w0["words"].T, o.words)  # [n_words][N] planes vs [N][n_words]
    del w0
    g.step(1)
    o.step(1)
    r = g.readback(state=False, words=True, ids=True)
    g.close()
    assert np.array_equal(r["ids"], o.ids)
    qt = quanta(oracle, sc, sch)[None]
    dmax, ndiff = 0.0, 0
    N = o.words.shape[0]
    for a in range(0, N, block):  # compare decoded blocks (the full arrays are tens of GB)
        mine = oracle.decode_state(o.cd, np.ascontiguousarray(r["words"][:, a:a + block].T), threaded=True)
        theirs = oracle.decode_state(o.cd, o.words[a:a + block], threaded=True)
        d = np.abs(mine - theirs) / qt
        dmax = max(dmax, float(d.max()))
        ndiff += int((d > 0).sum())
    return dmax, ndiff / (N * qt.shape[1])


@pytest.mark.parametrize("spec", [False, True], ids=["library", "specialized"])
def test_cubes_full_size_one_step(q, oracle, spec):
    # the benchmark's scheme (the cached second-order scheme) and kernel
    from paper_2207_04658_b300 import autoquant, scenes
    sc, s0 = scenes.cubes3d_scene(resort_every=20)  # as bench.py runs it
    assert s0.shape[0] == 8_192_000
    cached = autoquant.load_cubes3d_scheme(0.01)
    scheme = cached["scheme"] if cached is not None else autoquant.cubes3d_scheme(0.01)[0]
    dmax, frac = one_step_parity(q, oracle, sc, s0, scheme, spec=spec)
    assert dmax <= 2.0 and frac < 1e-3, (dmax, frac)


@pytest.mark.parametrize("dither,spec", [(True, False), (False, False), (True, True)])
def test_dambreak_full_size_one_step(q, oracle, dither, spec):
    from paper_2207_04658_b300 import scenes
    sc, s0 = scenes.dambreak3d_scene()
    assert s0.shape[0] == 2 ** 27
    sc = dict(sc, dither=dither)
    sch = scenes.fixed_scheme_3d("fluid", C=(16, -2048.0, 2048.0))
    dmax, frac = one_step_parity(q, oracle, sc, s0, sch, spec=spec)
    assert dmax <= 2.0 and frac < 1e-3, (dmax, frac)
