"""The C ABI library loads, exports every entry point include/qmpm.h declares, and its
host-only parts (record layout, scheme solve) agree with the oracle.  No GPU needed:
only pure-host entry points are called."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_functions():
    names = set()
    for path in HEADERS:
        text = open(path).read()
        names |= set(re.findall(r"^\s*(?:int|const char \*)\s*(qmpm_\w+)\s*\(", text, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def q():
    from paper_2207_04658_b300 import build, qmpm
    build.build()
    qmpm.lib()
    return qmpm


def test_library_exports_every_declared_symbol(q):
    names = declared_functions()
    assert "qmpm_init" in names and "qmpm_scheme_solve" in names and len(names) >= 12
    L = ct.CDLL(q.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols(q):
    bound = {n for n, _, _ in q._SIGNATURES + q.OPTIONAL_SIGNATURES}
    assert set(declared_functions()) <= bound


CASES = [(2, "neohookean"), (2, "fluid"), (3, "corotated"), (3, "fluid")]


@pytest.mark.parametrize("dim,material", CASES)
def test_layout_matches_oracle(q, oracle, dim, material):
    gen = np.random.default_rng(dim * 7 + len(material))
    for trial in range(50):
        bits = [int(b) for b in gen.integers(1, 25, 4)]
        cont = [int(c) for c in gen.choice([0, 32, 64], 4)]
        scheme = {n: dict(bits=bits[h], frac=10, offset=-5, container=cont[h])
                  for h, n in enumerate(["x", "v", "C", "J" if material == "fluid" else "F"])}
        s = q.make_scheme_struct(scheme, dim, material)
        fields = oracle.comp_fields(dim, material)
        pos, nw = oracle.layout(dim, material, [bits[h] for h in fields], cont)
        assert s.n_words == nw
        assert [s.bitpos[c] for c in range(len(fields))] == pos


def test_layout_rejects_bad_schemes(q):
    base = {n: dict(bits=16, frac=10, offset=0) for n in ["x", "v", "C", "F"]}
    for field, key, val in [("x", "bits", 25), ("v", "bits", 0), ("C", "offset", 2 ** 24),
                            ("F", "container", 48)]:
        bad = {k: dict(v) for k, v in base.items()}
        bad[field][key] = val
        with pytest.raises(q.QmpmError) as ei:
            q.make_scheme_struct(bad, 3, "corotated")
        assert ei.value.code == -3
    with pytest.raises(q.QmpmError):
        q.make_scheme_struct(base, 4, "corotated")


@pytest.mark.parametrize("mode,rounding", [("error", "paper"), ("error", "exact"),
                                           ("memory", "paper"), ("memory", "exact")])
def test_scheme_solve_matches_oracle(q, oracle, mode, rounding):
    gen = np.random.default_rng(len(mode) * 10 + len(rounding))
    for trial in range(20):
        H = int(gen.integers(1, 6))
        P = gen.integers(1000, 100000, H).astype(float)
        g = 10.0 ** gen.uniform(-6, 2, H)
        lo = gen.uniform(-5, 0, H)
        hi = lo + 10.0 ** gen.uniform(-1, 1.5, H)
        z = float(10.0 ** gen.uniform(-2, 3))
        eps = float(10.0 ** gen.uniform(-3, -1)) if mode == "error" else float(gen.uniform(0.3, 0.7))
        a = q.qmpm_scheme_solve(P, g, lo, hi, z, eps, mode=mode, rounding=rounding)
        b = oracle.scheme_solve(P, g, lo, hi, z, eps, mode=mode, rounding=rounding)
        assert a["bits"] == b["bits"] and a["frac"] == b["frac"] and a["offset"] == b["offset"]
        assert a["bits_paper"] == b["bits_paper"]
        assert np.allclose(a["delta_cont"], b["delta_cont"], rtol=1e-12)
        assert a["pred_err"] == pytest.approx(b["pred_err"], rel=1e-12)


def test_scheme_solve_rejects_bad_input(q):
    with pytest.raises(q.QmpmError):
        q.qmpm_scheme_solve([], [], [], [], 1.0, 0.01)
    with pytest.raises(q.QmpmError):
        q.qmpm_scheme_solve([1.0], [1.0], [0.0], [1.0], 1.0, 0.0)


def test_missing_library_fails_loudly(monkeypatch, q):
    from paper_2207_04658_b300 import qmpm as qm
    monkeypatch.setattr(qm, "_lib", None)
    monkeypatch.setattr(qm, "LIB_PATH", "/nonexistent/libqmpm.so")
    with pytest.raises(ImportError):
        qm.lib()


@pytest.mark.parametrize("case", ["cap", "refine", "margin", "all"])
def test_scheme_solve_options_match_oracle(q, oracle, case):
    gen = np.random.default_rng({"cap": 1, "refine": 2, "margin": 3, "all": 4}[case])
    for trial in range(40):
        H = int(gen.integers(2, 5))
        P = gen.integers(1000, 100000, H).astype(float)
        g = 10.0 ** gen.uniform(-4, 4, H)
        lo = gen.uniform(-5, 0, H)
        hi = lo + 10.0 ** gen.uniform(-1, 1.5, H)
        z = float(10.0 ** gen.uniform(-1, 2))
        eps = float(10.0 ** gen.uniform(-5, -1))
        kw = {}
        if case in ("cap", "all"):
            kw["max_bits"] = int(gen.integers(6, 20))
        if case in ("refine", "all"):
            kw["beta"] = list(gen.normal(0, 1, H) * 10.0 ** gen.uniform(0, 5, H))
        if case in ("margin", "all"):
            h = int(gen.integers(0, H))
            kw["margins"] = {h: (int(gen.integers(0, H)), float(10.0 ** gen.uniform(0, 3)))}
        a = q.qmpm_scheme_solve(P, g, lo, hi, z, eps, **kw)
        b = oracle.scheme_solve(P, g, lo, hi, z, eps, **kw)
        for key in ("bits", "frac", "offset", "capped_mask", "refined"):
            assert a[key] == b[key], (case, trial, key, a[key], b[key], kw)
        for key in ("pred_err", "pred_bias", "pred_var_dither", "total_bits"):
            assert a[key] == pytest.approx(b[key], rel=1e-12, abs=1e-300), (case, key)


def test_scheme_solve_options_reject_bad_input(q):
    with pytest.raises(q.QmpmError):
        q.qmpm_scheme_solve([1.0, 1.0], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0], 1.0, 0.01, max_bits=-1)
    with pytest.raises(q.QmpmError):
        q.qmpm_scheme_solve([1.0, 1.0], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0], 1.0, 0.01, margins={0: (5, 1.0)})


def test_step_host_stream_rejects_bad_arguments(q):
    # argument checks come before any CUDA call: no device needed
    for args in ((None, 1, 0, 0), (None, -1, 0, 0), (None, 1, 0, 65)):
        with pytest.raises(q.QmpmError) as ei:
            q.qmpm_step_host_stream(*args)
        assert ei.value.code == -1


def test_specialized_step_kernel_compiles_without_a_device(q):
    # the runtime compiler builds the scheme-specialised step kernel from the csrc/ sources
    # beside the library, for 2D/3D and every material, with and without statistics
    from paper_2207_04658_b300 import scenes
    cases = [(2, "neohookean", scenes.block2d_scheme()),
             (3, "corotated", scenes.fixed_scheme_3d("corotated")),
             (3, "fluid", scenes.fixed_scheme_3d("fluid", C=(16, -2048.0, 2048.0)))]
    for dim, material, scheme in cases:
        for stats, dither in ((False, True), (True, True), (False, False)):
            sec, nbytes = q.qmpm_specialize_compile(dim, material, scheme, stats, dither)
            assert nbytes > 10000 and sec >= 0.0
    # a second request returns the cached build
    first = q.qmpm_specialize_compile(3, "fluid", cases[2][2], False)
    assert q.qmpm_specialize_compile(3, "fluid", cases[2][2], False) == first


def test_specialize_compile_rejects_bad_input(q):
    # FP32 state (no scheme) compiles the kernel with its word count as the constant
    sec, nbytes = q.qmpm_specialize_compile(3, "corotated", None)
    assert nbytes > 10000
    with pytest.raises(q.QmpmError) as ei:
        q.qmpm_specialize_compile(4, "corotated", None)
    assert ei.value.code == -1
    with pytest.raises(q.QmpmError):
        q.qmpm_step_kernel_info(None)
