"""The C-ABI library builds, loads and exports every entry point that
include/xlmimo.h declares; argument validation rejects bad calls before any
device work (these calls never touch a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            syms |= set(re.findall(r"\b(xlmimo_[a-z0-9_]+)\s*\(", text))
    return syms


@pytest.fixture(scope="module")
def xl():
    from paper_2503_18118_gb300 import xlmimo
    xlmimo.lib()
    return xlmimo


def test_exports_every_declared_symbol(xl):
    syms = declared_symbols()
    assert {"xlmimo_channel_gram", "xlmimo_corr_closed_form", "xlmimo_beamform", "xlmimo_sumrate",
            "xlmimo_capacity_sweep"} <= syms
    L = xl.lib()
    for s in sorted(syms):
        assert hasattr(L, s), s
    assert set(xl.EXPORTS) >= syms


def test_version(xl):
    assert xl.xlmimo_version() >> 16 == 1


def test_invalid_arguments_rejected_on_host(xl):
    L = xl.lib()
    arr = xl.array(256, 0.01)
    dummy = ctypes.c_void_p(16)
    # K out of range
    assert L.xlmimo_channel_gram(ctypes.byref(arr), dummy, 65, 1, xl.F32, dummy, None) == 1
    assert b"K must be" in L.xlmimo_last_error()
    assert L.xlmimo_channel_gram(ctypes.byref(arr), dummy, 0, 1, xl.F32, dummy, None) == 1
    # bad geometry
    bad = xl.array(0, 0.01)
    assert L.xlmimo_channel_gram(ctypes.byref(bad), dummy, 4, 1, xl.F32, dummy, None) == 1
    bad = xl.array(16, -1.0)
    assert L.xlmimo_corr_closed_form(ctypes.byref(bad), dummy, 4, 1, dummy, None) == 1
    bad = xl.array(16, 0.01, model=7)
    assert L.xlmimo_channel_gram(ctypes.byref(bad), dummy, 4, 1, xl.F32, dummy, None) == 1
    # unknown precision, scheme, power mode
    assert L.xlmimo_channel_gram(ctypes.byref(arr), dummy, 4, 1, 9, dummy, None) == 1
    assert L.xlmimo_beamform(dummy, None, dummy, dummy, 4, 1, 5, 0, dummy, dummy, None, None) == 1
    assert L.xlmimo_beamform(dummy, None, dummy, dummy, 4, 1, 0x400, 0, dummy, dummy, None, None) == 1
    assert L.xlmimo_beamform(dummy, None, dummy, dummy, 4, 1, 5 | xl.MISMATCH_FP32, 0, dummy, dummy, None, None) == 1
    assert L.xlmimo_beamform(dummy, None, dummy, dummy, 4, 1, 0, 3, dummy, dummy, None, None) == 1
    # NULL buffers
    assert L.xlmimo_channel_gram(ctypes.byref(arr), None, 4, 1, xl.F32, dummy, None) == 1
    assert L.xlmimo_sumrate(None, 4, 3, dummy, None, None) == 1
    # saturation threshold outside (0, 1)
    assert L.xlmimo_saturation(dummy, 4, 1, 1.0, 0.01, dummy, None) == 1
    d = xl.UserDist(xl.DIST_RECT, 0, 2.0, 1.0, 0.0, 1.0)
    out = (ctypes.c_double * 6)()
    assert L.xlmimo_saturation_analytic(ctypes.byref(d), 4, 0.9, 0.01, out, None) == 1


def test_empty_batch_is_a_no_op(xl):
    L = xl.lib()
    arr = xl.array(256, 0.01)
    assert L.xlmimo_channel_gram(ctypes.byref(arr), None, 4, 0, xl.F32, None, None) == 0
    assert L.xlmimo_corr_closed_form(ctypes.byref(arr), None, 4, 0, None, None) == 0
    assert L.xlmimo_beamform(None, None, None, None, 4, 0, 0, 0, None, None, None, None) == 0
    assert L.xlmimo_saturation(None, 4, 0, 0.9, 0.01, None, None) == 0


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle and the binding has no CPU path."""
    pkg = os.path.join(ROOT, "paper_2503_18118_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_surrogate_entries_validate_on_host(xl):
    L = xl.lib()
    dummy = ctypes.c_void_p(16)
    arr = xl.array(1024, 0.01)
    assert L.xlmimo_pair_features(ctypes.byref(arr), dummy, 1, 1, 0, None, None, dummy, None, None, None) == 1
    assert L.xlmimo_pair_features(ctypes.byref(arr), dummy, 4, 1, 0, None, None, dummy, dummy, None, None) == 1
    assert b"targets need" in L.xlmimo_last_error()
    assert L.xlmimo_pair_features(ctypes.byref(arr), dummy, 4, 1, 3, None, None, dummy, None, None, None) == 1
    assert L.xlmimo_pair_features(ctypes.byref(arr), None, 4, 0, 0, None, None, None, None, None, None) == 0
    assert L.xlmimo_corr_closed_form_aperture(ctypes.byref(arr), dummy, 4, 1, 3, dummy, None) == 1
    assert L.xlmimo_corr_closed_form_aperture(ctypes.byref(arr), None, 4, 0, 2, None, None) == 0
    assert L.xlmimo_mlp_adam(dummy, dummy, dummy, dummy, 0, 1e-3, 0.9, 0.999, 1e-8, None) == 1
    assert L.xlmimo_mlp_adam(dummy, dummy, dummy, dummy, 1, 1e-3, 1.0, 0.999, 1e-8, None) == 1
    assert L.xlmimo_mlp_forward(dummy, dummy, -1, dummy, None, None) == 1
    assert L.xlmimo_mlp_forward(dummy, dummy, 0, dummy, None, None) == 0
    assert L.xlmimo_mlp_pack(dummy, ctypes.c_void_p(24), None) == 1
    assert b"16-byte" in L.xlmimo_last_error()
    assert L.xlmimo_surrogate_gram(ctypes.byref(arr), dummy, 4, 1, 0, ctypes.c_void_p(8), dummy, None) == 1
    assert L.xlmimo_surrogate_gram(ctypes.byref(arr), dummy, 65, 1, 0, dummy, dummy, None) == 1
    assert L.xlmimo_surrogate_gram(ctypes.byref(arr), dummy, 4, 1, 7, dummy, dummy, None) == 1
    assert L.xlmimo_surrogate_gram(ctypes.byref(arr), None, 4, 0, 0, None, None, None) == 0
    assert L.xlmimo_mlp_train_step(dummy, dummy, dummy, dummy, 1, 1e-3, dummy, dummy, None, 0, dummy, dummy,
                                   dummy, None, None) == 1
    # workspace: two [M][256] slabs plus one [257][256] partial per 512 rows
    assert L.xlmimo_mlp_work_floats(0) == 0
    # dZ slabs, four 256-row weight-gradient slices, the packed BF16 weights of the three 256 x 256 layers
    assert L.xlmimo_mlp_work_floats(1000) == 2 * 1000 * 256 + 4 * 257 * 256 + 3 * 2 * 4 * 256 * 64 * 2 // 4


def test_capacity_bounds_validates_on_host(xl):
    L = xl.lib()
    dummy = ctypes.c_void_p(16)
    arr = xl.array(1024, 0.01)
    assert L.xlmimo_capacity_bounds(ctypes.byref(arr), dummy, 0, 1, 1.0, dummy, None) == 1
    assert L.xlmimo_capacity_bounds(ctypes.byref(arr), dummy, xl.MAX_BOUNDS_USERS + 1, 1, 1.0, dummy, None) == 1
    assert L.xlmimo_capacity_bounds(ctypes.byref(arr), dummy, 8, 1, -1.0, dummy, None) == 1
    assert L.xlmimo_capacity_bounds(ctypes.byref(arr), dummy, 8, 1, float("nan"), dummy, None) == 1
    assert L.xlmimo_capacity_bounds(ctypes.byref(arr), None, 8, 1, 1.0, dummy, None) == 1
    assert L.xlmimo_capacity_bounds(ctypes.byref(arr), None, 8, 0, 1.0, None, None) == 0


def test_gram_ura_validates_on_host(xl):
    L = xl.lib()
    dummy = ctypes.c_void_p(16)
    arr = xl.array(1024, 0.01)
    assert L.xlmimo_channel_gram_ura(ctypes.byref(arr), 0, dummy, 8, 1, 1, dummy, None) == 1
    assert L.xlmimo_channel_gram_ura(ctypes.byref(arr), xl.MAX_URA_ROWS + 1, dummy, 8, 1, 1, dummy, None) == 1
    big = xl.array(1 << 30, 0.01)
    assert L.xlmimo_channel_gram_ura(ctypes.byref(big), 1025, dummy, 8, 1, 1, dummy, None) == 1
    assert L.xlmimo_channel_gram_ura(ctypes.byref(arr), 4, dummy, 8, 1, 9, dummy, None) == 1
    assert L.xlmimo_channel_gram_ura(ctypes.byref(arr), 4, None, 8, 1, 1, dummy, None) == 1
    assert L.xlmimo_channel_gram_ura(ctypes.byref(arr), 4, dummy, xl.MAX_USERS + 1, 1, 1, dummy, None) == 1
    assert L.xlmimo_channel_gram_ura(ctypes.byref(arr), 4, None, 8, 0, 1, None, None) == 0


def test_shutdown_without_state_is_a_no_op(xl):
    assert xl.lib().xlmimo_shutdown() == 0


def test_mc_step_validates_on_host(xl):
    L = xl.lib()
    dummy = 16
    good = dict(arr=xl.array(1024, 0.01), prec=xl.F32, scheme=xl.MMSE, cf_scheme=xl.ZF, power_mode=xl.POWER_RXSNR,
                K=8, B=4, chunks=0, reserved=0, t=0.9)
    ptrs = ("users", "power", "noise", "gram", "gram_cf", "sinr", "sinr_cf", "status", "status_cf", "rate", "rate_cf",
            "sat")

    def job(**over):
        j = xl.McBatch(**{**good, **over})
        for n in ptrs:
            setattr(j, n, dummy)
        return j

    assert L.xlmimo_mc_step(None, None) == 1
    for over in (dict(K=0), dict(K=65), dict(B=-1), dict(prec=9), dict(scheme=7), dict(cf_scheme=-2),
                 dict(power_mode=5), dict(chunks=65), dict(reserved=1), dict(t=1.0), dict(t=-0.5),
                 dict(arr=xl.array(0, 0.01))):
        assert L.xlmimo_mc_step(ctypes.byref(job(**over)), None) == 1, over
    j = job()
    j.sat = None
    assert L.xlmimo_mc_step(ctypes.byref(j), None) == 1  # t > 0 needs the saturation output
    j = job()
    j.gram_cf = None
    assert L.xlmimo_mc_step(ctypes.byref(j), None) == 1  # the closed-form path needs its buffers
    assert L.xlmimo_mc_step(ctypes.byref(job(B=0)), None) == 0


def test_capacity_sweep_and_batch_plan_validate_on_host(xl):
    L = xl.lib()
    res = xl.SweepResult()
    assert L.xlmimo_capacity_sweep(None, ctypes.byref(res), None) == 1
    cfg = xl.SweepCfg(wavelength=0.01, spacing=0.005, beta0=1.0, model=xl.FSPL_USW, prec=xl.F32, n_count=0,
                      snr_count=0, K=8, B=4, t=0.9, ref_x=10.0)
    assert L.xlmimo_capacity_sweep(ctypes.byref(cfg), ctypes.byref(res), None) == 1  # no n_list, snr_db or users
    geo = xl.array(1024, 0.01)
    insts = (xl.Inst * 1)(xl.Inst(1024, 8, xl.ZF, 0, 0, 1.0))
    plan = ctypes.c_void_p()
    assert L.xlmimo_batch_plan_create(None, insts, 1, xl.BF16X3, None, ctypes.byref(plan), None) == 1
    assert L.xlmimo_batch_plan_create(ctypes.byref(geo), insts, 0, xl.BF16X3, None, ctypes.byref(plan), None) == 1
    assert L.xlmimo_batch_plan_create(ctypes.byref(geo), insts, 1, xl.F32, None, ctypes.byref(plan), None) == 1
    bad = (xl.Inst * 1)(xl.Inst(1024, 65, xl.ZF, 0, 0, 1.0))
    assert L.xlmimo_batch_plan_create(ctypes.byref(geo), bad, 1, xl.BF16X3, None, ctypes.byref(plan), None) == 1
    assert L.xlmimo_batch_plan_set_tiling(None, 8192, 2, 32, 1, None) == 1


def test_binding_constants_match_header(xl):
    """The binding's size limits are the header's."""
    text = open(os.path.join(ROOT, "include", "xlmimo.h")).read()
    defs = dict(re.findall(r"#define\s+XLMIMO_([A-Z0-9_]+)\s+(\d+)", text))
    assert int(defs["NOALLOC_SCRATCH_MIB"]) == xl.NOALLOC_SCRATCH_MIB
    assert int(defs["MAX_USERS"]) == xl.MAX_USERS
    assert int(defs["PLAN_INFO_LEN"]) == xl.PLAN_INFO_LEN
    assert int(re.search(r"#define\s+XLMIMO_MISMATCH_FP32\s+0x([0-9a-fA-F]+)", text).group(1), 16) == xl.MISMATCH_FP32
    assert int(re.search(r"#define\s+XLMIMO_FACTOR_FF\s+0x([0-9a-fA-F]+)", text).group(1), 16) == xl.FACTOR_FF


def test_remaining_entries_validate_on_host(xl):
    """Every entry point rejects bad arguments before any device work: the
    allocation-free Gram, the timed bounds, the rate and saturation calls, the
    batch-plan calls, the network's training calls and the pipe probe."""
    L = xl.lib()
    dummy = ctypes.c_void_p(16)
    arr = xl.array(1024, 0.01)
    # allocation-free Gram: K range, precision, NULL buffers; the tensor-core
    # precisions are valid requests this entry point does not serve
    for K in (0, xl.MAX_USERS + 1):
        assert L.xlmimo_channel_gram_noalloc(ctypes.byref(arr), dummy, K, 1, xl.F32, dummy, None) == 1
    assert L.xlmimo_channel_gram_noalloc(ctypes.byref(arr), dummy, 4, -1, xl.F32, dummy, None) == 1
    assert L.xlmimo_channel_gram_noalloc(ctypes.byref(arr), dummy, 4, 1, 9, dummy, None) == 1
    assert L.xlmimo_channel_gram_noalloc(ctypes.byref(arr), dummy, 4, 1, xl.BF16X3, dummy, None) == 6
    assert L.xlmimo_channel_gram_noalloc(ctypes.byref(arr), None, 4, 1, xl.F64, dummy, None) == 1
    assert L.xlmimo_channel_gram_noalloc(ctypes.byref(arr), None, 4, 0, xl.F64, None, None) == 0
    # timed bounds: the phase times are required
    assert L.xlmimo_capacity_bounds_timed(ctypes.byref(arr), dummy, 8, 1, 1.0, dummy, None, None) == 1
    assert b"phase_ms" in L.xlmimo_last_error()
    # sum rate and per-trial saturation
    assert L.xlmimo_sumrate(dummy, 0, 1, dummy, None, None) == 1
    assert L.xlmimo_sumrate(dummy, 4, -1, dummy, None, None) == 1
    assert L.xlmimo_sumrate(dummy, 4, 1, None, None, None) == 1
    assert L.xlmimo_sumrate(None, 4, 0, None, None, None) == 0
    for t, spacing in ((0.0, 0.01), (0.9, 0.0), (0.9, float("inf")), (float("nan"), 0.01)):
        assert L.xlmimo_saturation(dummy, 4, 1, t, spacing, dummy, None) == 1, (t, spacing)
    assert L.xlmimo_saturation(dummy, 4, 1, 0.9, 0.01, None, None) == 1
    # analytic saturation: descriptor, ranges, K, NULL output
    out = (ctypes.c_double * 6)()
    rect = xl.UserDist(xl.DIST_RECT, 0, 1.0, 10.0, -7.5, 7.5)
    assert L.xlmimo_saturation_analytic(None, 4, 0.9, 0.01, out, None) == 1
    assert L.xlmimo_saturation_analytic(ctypes.byref(rect), 4, 0.9, 0.01, None, None) == 1
    assert L.xlmimo_saturation_analytic(ctypes.byref(rect), 0, 0.9, 0.01, out, None) == 1
    assert L.xlmimo_saturation_analytic(ctypes.byref(rect), 4, 0.9, -0.01, out, None) == 1
    for bad in (xl.UserDist(xl.DIST_RECT, 1, 1.0, 10.0, -7.5, 7.5), xl.UserDist(2, 0, 1.0, 10.0, -7.5, 7.5),
                xl.UserDist(xl.DIST_RECT, 0, 0.0, 10.0, -7.5, 7.5), xl.UserDist(xl.DIST_RECT, 0, 1.0, 10.0, 7.5, -7.5),
                xl.UserDist(xl.DIST_POLAR, 0, 3.0, 30.0, -1.0, 1.6)):
        assert L.xlmimo_saturation_analytic(ctypes.byref(bad), 4, 0.9, 0.01, out, None) == 1
    # batch plans: a NULL plan is refused, and destroying it is a no-op
    info = (ctypes.c_int64 * xl.PLAN_INFO_LEN)()
    assert L.xlmimo_batch_run(None, dummy, dummy, 0, dummy, dummy, dummy, dummy, None) == 1
    assert L.xlmimo_batch_plan_info(None, info) == 1
    assert L.xlmimo_batch_plan_destroy(None) == 0
    # network training calls
    assert L.xlmimo_mlp_loss(dummy, dummy, None, -1, dummy, dummy, None) == 1
    assert L.xlmimo_mlp_loss(dummy, None, None, 4, dummy, dummy, None) == 1
    assert L.xlmimo_mlp_loss(None, None, None, 0, None, None, None) == 0
    assert L.xlmimo_mlp_backward(dummy, dummy, dummy, dummy, -1, dummy, dummy, None) == 1
    assert L.xlmimo_mlp_backward(None, dummy, dummy, dummy, 4, dummy, dummy, None) == 1
    assert L.xlmimo_mlp_backward(dummy, dummy, dummy, dummy, 4, dummy, ctypes.c_void_p(20), None) == 1
    assert b"16-byte" in L.xlmimo_last_error()
    for step, lr, b1, b2, eps in ((1, 1e-3, 0.9, 1.0, 1e-8), (1, 1e-3, 0.9, 0.999, 0.0), (1, -1.0, 0.9, 0.999, 1e-8)):
        assert L.xlmimo_mlp_adam(dummy, dummy, dummy, dummy, step, lr, b1, b2, eps, None) == 1
    assert L.xlmimo_mlp_adam(None, dummy, dummy, dummy, 1, 1e-3, 0.9, 0.999, 1e-8, None) == 1
    # a training step checks Adam's step and rate before it enqueues its forward pass
    step_args = lambda step, lr, work=dummy: (dummy, dummy, dummy, dummy, step, lr, dummy, dummy, None, 4, dummy,
                                              dummy, work, None, None)
    assert L.xlmimo_mlp_train_step(*step_args(0, 1e-3)) == 1
    assert b"step" in L.xlmimo_last_error()
    assert L.xlmimo_mlp_train_step(*step_args(1, float("nan"))) == 1
    assert L.xlmimo_mlp_train_step(*step_args(1, 1e-3, ctypes.c_void_p(20))) == 1
    assert L.xlmimo_mlp_forward(None, dummy, 4, dummy, None, None) == 1
    # pipe probe
    res = (ctypes.c_double * 2)()
    for pipe in (-1, 3):
        assert L.xlmimo_measure_pipe(pipe, res, None) == 1
    assert L.xlmimo_measure_pipe(0, None, None) == 1
    # pair features: K range, base, weights without the closed form
    assert L.xlmimo_pair_features(ctypes.byref(arr), dummy, xl.MAX_USERS + 1, 1, 0, None, None, dummy, None, None,
                                  None) == 1
    assert L.xlmimo_pair_features(ctypes.byref(arr), dummy, 4, 1, -1, None, None, dummy, None, None, None) == 1
    assert L.xlmimo_pair_features(ctypes.byref(arr), dummy, 4, 1, 0, None, None, dummy, None, dummy, None) == 1
    assert b"weights need" in L.xlmimo_last_error()


def test_readme_example_uses_the_binding(xl):
    """Every binding name and workload field the README's Python example uses
    exists (the calls themselves need a GPU)."""
    from paper_2503_18118_gb300 import inputs
    text = open(os.path.join(ROOT, "README.md")).read()
    src = text.split("```python")[1].split("```")[0]
    for name in set(re.findall(r"\bxl\.([A-Za-z_0-9]+)", src)):
        assert hasattr(xl, name), name
    for name in set(re.findall(r"\bwl\.([A-Za-z_0-9]+)", src)):
        assert hasattr(inputs.HEADLINE, name), name


def test_binding_refuses_host_tensors(xl):
    """The binding passes device pointers only: host tensors, wrong dtypes and
    shapes are refused before the library is called."""
    torch = pytest.importorskip("torch")
    arr = xl.array(256, 0.01)
    with pytest.raises(TypeError):
        xl.xlmimo_channel_gram(arr, torch.zeros((2, 4, 2), dtype=torch.float64))
    with pytest.raises(TypeError):
        xl.xlmimo_corr_closed_form(arr, torch.zeros((2, 4, 2), dtype=torch.float32))
    with pytest.raises(TypeError):
        xl.xlmimo_saturation(torch.zeros((2, 4, 2), dtype=torch.float64), 0.9, 0.005)


def test_build_tracks_every_source_and_header():
    """The library is rebuilt when any kernel source, kernel header or the C
    interface header changes (its staleness check covers all of them)."""
    import glob
    from paper_2503_18118_gb300 import build as b
    deps = set(b._deps())
    csrc = os.path.join(ROOT, "paper_2503_18118_gb300", "csrc")
    want = set(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
               glob.glob(os.path.join(ROOT, "include", "*.h")))
    assert want and want <= deps
    assert set(b._sources()) == set(glob.glob(os.path.join(csrc, "*.cu")))
