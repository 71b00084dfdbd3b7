"""The shell-MAC autotuner: both kernels agree with the FP64 oracle at every
slice count, and the tuner's choices are reported and persisted."""
import numpy as np
import pytest

import oracle
import paper_1502_02294_gb300 as lc
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_L2, FP32_MAX, BF16_L2 = 1e-5, 1e-4, 5e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()
    oracle.build()


def _fields(w, steps, check):
    plan = lc.Plan.from_workload(w)
    out = {}
    for s in steps:
        pos, lum = w.cat.active(s)
        plan.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        if s in check:
            out[s] = plan.field(s).cpu().numpy()
    plan.close()
    return out


def _errors(J, ref):
    J = np.asarray(J, dtype=np.float64)
    a = np.abs(ref)
    ulp = np.exp2(np.floor(np.log2(np.maximum(a, np.finfo(np.float32).tiny))) - 23)
    rel = np.linalg.norm(J - ref) / np.linalg.norm(ref)
    mx = np.maximum(np.abs(J - ref) - 2.0 * ulp, 0.0).max() / a.mean()
    return rel, mx


@pytest.mark.parametrize("history", [synth.HISTORY_FP32, synth.HISTORY_BF16])
@pytest.mark.parametrize("variant", ["gather", "bulk", "ws", "ws2"])
def test_forced_variant_matches_oracle_every_slice_count(monkeypatch, variant, history):
    # c1 (32^3, 8 steps): slice counts 1..8 cover a partial Ghat block and
    # fewer slices than pipeline stages
    monkeypatch.setenv("LC_MAC_VARIANT", variant)
    w = synth.config("c1")
    w.history = history
    P = oracle.Problem.from_workload(w)
    out = _fields(w, range(8), set(range(8)))
    for s, J in out.items():
        ref = oracle.field_for(P, w.cat, s)
        rel, mx = _errors(J, ref)
        if history == synth.HISTORY_FP32:
            assert rel <= FP32_L2 and mx <= FP32_MAX, (variant, s, rel, mx)
        else:
            assert rel <= BF16_L2, (variant, s, rel)


def test_forced_variants_agree_many_slices(monkeypatch):
    # 64^3 with 20 steps: up to 20 slices, more than two Ghat blocks
    w = synth.small(n=64, box=90.0, n_steps=20, n_src=300, subsamples=2, clustered=True, seed=4242)
    P = oracle.Problem.from_workload(w)
    res = {}
    for v in ("gather", "bulk", "ws", "ws2"):
        monkeypatch.setenv("LC_MAC_VARIANT", v)
        res[v] = _fields(w, range(20), {12, 19})
    for s in (12, 19):
        # every MAC kernel does the same arithmetic in the same order
        for v in ("bulk", "ws", "ws2"):
            assert np.array_equal(res["gather"][s], res[v][s]), (v, s)
        ref = oracle.field_for(P, w.cat, s)
        for v in ("gather", "bulk", "ws", "ws2"):
            rel, mx = _errors(res[v][s], ref)
            assert rel <= FP32_L2 and mx <= FP32_MAX, (v, s, rel, mx)


def test_choices_reported_and_persisted(monkeypatch, tmp_path):
    cache = tmp_path / "tune.txt"
    monkeypatch.delenv("LC_MAC_VARIANT", raising=False)
    monkeypatch.setenv("LC_AUTOTUNE_CACHE", str(cache))
    # 96^3 with a BF16 history: keys no other test tunes, so they are new here
    w = synth.small(n=96, box=120.0, n_steps=4, n_src=60, seed=515, history=synth.HISTORY_BF16)
    _fields(w, range(4), {3})
    rep = lc.autotune_report()
    mine = {k: v for k, v in rep.items() if "/N96/bf16/" in k}
    assert mine and set(mine.values()) <= {"gather", "bulk", "ws", "ws2"}
    lines = cache.read_text().split()
    assert any("/N96/bf16/" in t for t in lines)


@pytest.mark.parametrize("history", [synth.HISTORY_FP32, synth.HISTORY_BF16])
def test_large_grid_8_column_tiles_against_oracle(monkeypatch, history):
    # 384^3 (8-column x-pass tiles): every MAC kernel built at this size gives
    # the same field, which matches the oracle on sampled cells
    w = synth.small(n=384, box=300.0, n_steps=8, n_src=60, subsamples=2, clustered=True, seed=384,
                    z_start=16.0, z_end=15.0, history=history)
    res = {}
    for v in ("gather", "ws", "ws2"):
        monkeypatch.setenv("LC_MAC_VARIANT", v)
        res[v] = _fields(w, range(8), {7})[7]
    for v in ("ws", "ws2"):
        assert np.array_equal(res["gather"], res[v]), v
    P = oracle.Problem.from_workload(w)
    assert P.active_shells(7) >= 4
    pos, lum = w.cat.active(7)
    dense = np.floor(pos[np.argmax(lum)] / (w.box / w.n) + 0.5).astype(int) % w.n
    cells = synth.sample_cells(4242, w.n, 2000, dense_line_through=dense)
    ref = oracle.field_for(P, w.cat, 7, cells=cells)
    got = res["gather"].reshape(-1)[cells].astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= (FP32_L2 if history == synth.HISTORY_FP32 else BF16_L2), rel


def test_512_bf16_mac_kernels_agree(monkeypatch):
    # 512^3 BF16: the paired warp-specialised kernel equals the gather pass bit for bit
    w = synth.small(n=512, box=400.0, n_steps=8, n_src=40, subsamples=2, clustered=True, seed=512,
                    z_start=16.0, z_end=15.0, history=synth.HISTORY_BF16)
    res = {}
    for v in ("gather", "ws2"):
        monkeypatch.setenv("LC_MAC_VARIANT", v)
        res[v] = _fields(w, range(8), {7})[7]
    assert np.array_equal(res["gather"], res["ws2"])
    assert np.isfinite(res["ws2"]).all() and res["ws2"].max() > 0


@pytest.mark.parametrize("n", [256, 384, 512])
def test_fft_pass_forms_against_numpy_and_each_other(n):
    # both forms of the FFT passes (block-wide stages, one lane per column)
    # against numpy's FP64 transform, Parseval, and the round trip
    before = lc.fft_variant(n)
    rng = np.random.default_rng(n + 7)
    x = rng.standard_normal((n, n, n)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    ref = np.fft.rfftn(x.astype(np.float64))
    res = {}
    forms = (lc.FFT_STAGES, lc.FFT_LANES, lc.FFT_LANES3, lc.FFT_TMA, lc.FFT_TMA4) + (
        (lc.FFT_PLANE4,) if n == 256 else ())
    try:
        for v in forms:
            lc.fft_set_variant(n, v)
            assert lc.fft_variant(n) == v
            X = lc.fft_r2c(xt)
            Xn = X.cpu().numpy().astype(np.complex128)
            err = np.linalg.norm(Xn - ref) / np.linalg.norm(ref)
            assert err < 2e-6, (v, err)
            back = lc.fft_c2r(X).cpu().numpy()
            assert np.abs(back - x).max() < 1e-5 * np.abs(x).max(), v
            res[v] = Xn
    finally:
        lc.fft_set_variant(n, before)
    for v in forms[1:]:
        d = np.linalg.norm(res[lc.FFT_STAGES] - res[v]) / np.linalg.norm(ref)
        assert d < 2e-6, (v, d)
    # the same arithmetic under other tile schedules and copy engines
    assert np.array_equal(res[lc.FFT_LANES], res[lc.FFT_LANES3])
    assert np.array_equal(res[lc.FFT_LANES], res[lc.FFT_TMA])
    assert np.array_equal(res[lc.FFT_LANES], res[lc.FFT_TMA4])


def test_fft_pass_forms_give_oracle_fields():
    # a 256^3 field with each form of the passes against the FP64 oracle
    w = synth.small(n=256, box=200.0, n_steps=8, n_src=300, subsamples=2, clustered=True, seed=2561,
                    z_start=16.0, z_end=15.0, history=synth.HISTORY_FP32)
    P = oracle.Problem.from_workload(w)
    pos, lum = w.cat.active(7)
    dense = np.floor(pos[np.argmax(lum)] / (w.box / w.n) + 0.5).astype(int) % w.n
    cells = synth.sample_cells(2562, w.n, 1500, dense_line_through=dense)
    ref = oracle.field_for(P, w.cat, 7, cells=cells)
    before = lc.fft_variant(256)
    try:
        for v in (lc.FFT_STAGES, lc.FFT_LANES, lc.FFT_LANES3, lc.FFT_TMA, lc.FFT_TMA4, lc.FFT_PLANE4):
            lc.fft_set_variant(256, v)
            got = _fields(w, range(8), {7})[7].reshape(-1)[cells].astype(np.float64)
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= FP32_L2, (v, rel)
    finally:
        lc.fft_set_variant(256, before)


@pytest.mark.parametrize("n", [16, 32, 64, 96, 128, 192])
def test_plane_forms_against_numpy_and_each_other(n):
    # grids with plane kernels (z + y per x-plane in shared memory): the
    # staged plane kernels and the register (lanes) ones against numpy's FP64
    # transform, and the round trip; 16^3 has the staged form only
    before = lc.fft_variant(n)
    rng = np.random.default_rng(n + 11)
    x = rng.standard_normal((n, n, n)).astype(np.float32)
    x[3, 5, 7] += 50.0  # a bright cell, so the spectrum is not flat
    xt = torch.from_numpy(x).cuda()
    ref = np.fft.rfftn(x.astype(np.float64))
    forms = [lc.FFT_STAGES] + ([lc.FFT_LANES] if n >= 32 else [])
    res = {}
    try:
        for v in forms:
            lc.fft_set_variant(n, v)
            assert lc.fft_variant(n) == v
            X = lc.fft_r2c(xt)
            Xn = X.cpu().numpy().astype(np.complex128)
            err = np.linalg.norm(Xn - ref) / np.linalg.norm(ref)
            assert err < 2e-6, (v, err)
            back = lc.fft_c2r(X).cpu().numpy()
            assert np.abs(back - x).max() < 1e-5 * np.abs(x).max(), v
            # the inverse on a spectrum with non-Hermitian DC / Nyquist imaginary parts ignores them
            Y = X.clone()
            Y[0, 0, 0] += 3j
            Y[0, 0, n // 2] += 2j
            back2 = lc.fft_c2r(Y).cpu().numpy()
            assert np.abs(back2 - x).max() < 1e-5 * np.abs(x).max(), v
            res[v] = Xn
    finally:
        if before >= 0:
            lc.fft_set_variant(n, before)
    if len(forms) == 2:
        d = np.linalg.norm(res[lc.FFT_STAGES] - res[lc.FFT_LANES]) / np.linalg.norm(ref)
        assert d < 2e-6, d


@pytest.mark.parametrize("n,hist", [(64, synth.HISTORY_FP32), (128, synth.HISTORY_FP32), (96, synth.HISTORY_BF16),
                                    (192, synth.HISTORY_BF16)])
def test_plane_forms_give_oracle_fields(n, hist):
    w = synth.small(n=n, box=0.78125 * n, n_steps=6, n_src=250, subsamples=2, clustered=True, seed=1900 + n,
                    history=hist)
    P = oracle.Problem.from_workload(w)
    cells = synth.sample_cells(1901 + n, w.n, 2000)
    ref = oracle.field_for(P, w.cat, 5, cells=cells)
    before = lc.fft_variant(n)
    got = {}
    try:
        for v in (lc.FFT_STAGES, lc.FFT_LANES):
            lc.fft_set_variant(n, v)
            got[v] = _fields(w, range(6), {5})[5].reshape(-1)[cells].astype(np.float64)
            rel = np.linalg.norm(got[v] - ref) / np.linalg.norm(ref)
            assert rel <= (FP32_L2 if hist == synth.HISTORY_FP32 else BF16_L2), (v, rel)
    finally:
        lc.fft_set_variant(n, before)
