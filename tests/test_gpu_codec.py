"""Device codec vs the oracle: encode (Sec. 3.1 Eq. 3 with the dithered store of Sec. 5
Eq. 11), bit pack / bit struct placement (Sec. 7) and decode are bit-exact on identical
FP32 inputs.  Runs through the C ABI (qmpm_pack_f32 / qmpm_unpack_f32)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAT = {"neohookean": 0, "corotated": 1, "fluid": 2}


def field_names(material):
    return ["x", "v", "C", "J" if material == "fluid" else "F"]


SCHEMES = [
    # (dim, material, {field: (bits, frac, offset, container)})
    (2, "neohookean", {"x": (16, 16, 0, 0), "v": (16, 13, -32768, 0), "C": (16, 9, -32768, 0),
                       "F": (16, 15, 0, 0)}),
    (3, "corotated", {"x": (21, 21, 0, 64), "v": (13, 9, -4096, 0), "C": (11, 3, -1024, 0),
                      "F": (17, 16, -65536, 0)}),
    (3, "fluid", {"x": (20, 20, 0, 0), "v": (9, 5, -256, 32), "C": (14, 4, -8192, 64),
                  "J": (23, 21, 0, 32)}),
    (2, "fluid", {"x": (24, 24, 0, 32), "v": (1, 0, -1, 0), "C": (7, -2, -64, 0), "J": (5, 3, 4, 0)}),
    (3, "neohookean", {"x": (19, 19, 0, 0), "v": (24, 20, -8388608, 0), "C": (3, 1, -4, 0),
                       "F": (12, 10, -2048, 64)}),
]


def scheme_dict(material, spec):
    out = {}
    for name in field_names(material):
        b, f, o, c = spec[name]
        out[name] = dict(bits=b, frac=f, offset=o, container=c)
    return out


def random_values(gen, dim, material, scheme, N):
    fields = []
    for c in range(2 * dim + dim * dim + (1 if material == "fluid" else dim * dim)):
        fields.append(0 if c < dim else 1 if c < 2 * dim else 2 if c < 2 * dim + dim * dim else 3)
    names = field_names(material)
    vals = np.zeros((N, len(fields)), dtype=np.float32)
    for c, h in enumerate(fields):
        f = scheme[names[h]]
        d = 2.0 ** -f["frac"]
        lo = f["offset"] * d
        hi = (f["offset"] + 2 ** f["bits"]) * d
        span = hi - lo
        vals[:, c] = gen.uniform(lo - 0.05 * span, hi + 0.05 * span, N).astype(np.float32)
        # exact grid points and half-way points exercise the tie rule
        k = gen.integers(0, N, N // 20)
        vals[k, c] = ((f["offset"] + gen.integers(0, 2 ** f["bits"], len(k)) + 0.5 * gen.integers(0, 2, len(k))) * d).astype(np.float32)
    specials = [np.nan, np.inf, -np.inf, 0.0, -0.0, 1e30, -1e30, 1e-30]
    for i, v in enumerate(specials):
        vals[i % N, i % vals.shape[1]] = v
    return vals


@pytest.fixture(scope="module")
def q():
    import torch
    from paper_2207_04658_b300 import qmpm
    assert torch.cuda.is_available()
    qmpm.lib()
    return qmpm


@pytest.mark.parametrize("case", range(len(SCHEMES)))
@pytest.mark.parametrize("dither", [True, False])
def test_pack_unpack_bit_exact(q, oracle, case, dither):
    import torch
    dim, material, spec = SCHEMES[case]
    scheme = scheme_dict(material, spec)
    gen = np.random.default_rng(case * 2 + int(dither))
    N = 20_011  # ragged: not a multiple of the CTA size
    ld = N + 13
    vals = random_values(gen, dim, material, scheme, N)
    seed, step = 0x1234_5678_9ABC_DEF0 + case, 77 + case
    s = q.make_scheme_struct(scheme, dim, material)
    W = s.n_words
    d_vals = torch.from_numpy(vals).cuda()
    d_words = torch.zeros((W, ld), dtype=torch.int32, device="cuda")
    st = q.qmpm_stats_t()
    q.qmpm_pack_f32(dim, MAT[material], s, seed, dither, step, d_vals.data_ptr(), N,
                    d_words.data_ptr(), ld, st, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = d_words.cpu().numpy().view(np.uint32)[:, :N].T

    sc = dict(dim=dim, material=material, seed=seed, dither=dither)
    cd = oracle.make_codec(sc, scheme)
    assert cd.n_words == W
    ost = np.zeros(oracle.N_STATS, dtype=np.int64)
    want = oracle.encode_state(cd, vals.astype(np.float64), step, ost)
    mism = np.argwhere(got != want)
    assert mism.size == 0, f"{len(mism)} words differ, first at {mism[:3].tolist()}"
    assert list(st.saturations) == list(ost[0:4])
    assert list(st.round_ups) == list(ost[4:8])
    assert list(st.round_downs) == list(ost[8:12])

    d_out = torch.zeros((N, vals.shape[1]), dtype=torch.float32, device="cuda")
    q.qmpm_unpack_f32(dim, MAT[material], s, d_words.data_ptr(), N, ld, d_out.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    dec_gpu = d_out.cpu().numpy()
    dec_or = oracle.decode_state(cd, want).astype(np.float32)
    assert np.array_equal(dec_gpu.view(np.uint32), dec_or.view(np.uint32))


def test_dither_statistics_on_device(q, oracle):
    # Sec. 5: round-up probability equals the fractional part; 1e6 device draws
    import torch
    n = 1_000_000
    Y = 0.3
    scheme = scheme_dict("fluid", {"x": (12, 10, -512, 0), "v": (12, 10, -512, 0),
                                   "C": (12, 10, -512, 0), "J": (12, 10, -512, 0)})
    s = q.make_scheme_struct(scheme, 2, "fluid")
    vals = np.full((n, 9), (37 + Y) * 2.0 ** -10, dtype=np.float32)
    d_vals = torch.from_numpy(vals).cuda()
    d_words = torch.zeros((s.n_words, n), dtype=torch.int32, device="cuda")
    st = q.qmpm_stats_t()
    q.qmpm_pack_f32(2, 2, s, 99, True, 5, d_vals.data_ptr(), n, d_words.data_ptr(), n, st, 0)
    ups = sum(st.round_ups)
    downs = sum(st.round_downs)
    assert ups + downs == 9 * n
    sigma = math.sqrt(Y * (1 - Y) / (9 * n))
    assert abs(ups / (9 * n) - Y) < 4 * sigma
