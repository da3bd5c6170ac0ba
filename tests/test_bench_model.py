"""The roofline work model of bench.py (host arithmetic, no GPU): pruned
transform bytes by hand for a small grid, pair flops, and the per-stage /
path roofline fractions."""
import math

import bench


def test_fft_buffer_bytes_by_hand():
    """Mt = 2: padded grid 4 x 4 x 8, half spectrum 4 x 4 x 5, data region
    2 x 2 x 4 real values.  Forward: z lines of the 2 x 2 data columns (read 16
    reals, write 20 complex), y lines of the 2 data x planes over 5 kz (read
    2 x 5 x 2, write 2 x 5 x 4 complex), x lines over every (y, kz) (read
    4 x 5 x 2, write 4 x 5 x 4)."""
    e = 8
    byts, flops = bench.fft_buffer_work(2, e)
    c = 16
    z = 16 * e + 20 * c
    y = 20 * c + 40 * c
    x = 40 * c + 80 * c
    assert byts == z + y + x
    # 4 real lines of 8, 10 complex lines of 4 (y), 20 complex lines of 4 (x)
    assert math.isclose(flops, 4 * 2.5 * 8 * 3 + 10 * 5 * 4 * 2 + 20 * 5 * 4 * 2)


def test_fft_bytes_of_the_bench_grid():
    """At Mt = 320 one buffer's pruned passes move about 11 GB (z 1.6, y 3.2,
    x 6.3 GB), so the 7 forward and 4 inverse transforms of the bench
    workload move about 77 and 44 GB."""
    byts, _ = bench.fft_buffer_work(320, 8)
    assert 10.9e9 < byts < 11.2e9
    assert 76e9 < 7 * byts < 78e9


def test_pair_flops():
    # one unordered free pair (2 ordered), no images
    assert bench.pair_flops(2, 0, 0) == bench.FLOPS_RADIAL + 2 * bench.FLOPS_FREE_DIR
    # a target's own image only
    assert bench.pair_flops(0, 1, 1) == bench.FLOPS_RADIAL + bench.FLOPS_IMAGE_DIR
    # one unordered image pair (2 ordered) between different particles
    assert bench.pair_flops(0, 2, 0) == bench.FLOPS_RADIAL + 2 * bench.FLOPS_IMAGE_DIR


def test_pair_flops_split_by_kind():
    # counts (ordered free, ordered image, own images) by cut-off, as the
    # count-only plan would return them; nothing here touches a GPU
    pc = bench.PairCounter(None, 0, None, None)
    pc.cache = {0.05: (1000, 300, 10), 0.02: (100, 40, 6), 0.004: (8, 4, 2)}
    total = bench.pair_flops(1000, 300, 10)
    inner = bench.pair_flops(100, 40, 6)
    mid = bench.pair_flops(8, 4, 2)
    prm = {"rc": 0.05, "rc64": 0.02, "rcmid": 0.004}
    assert pc.flops("mixed", prm) == {"fp32": total}
    assert pc.flops("plain", prm) == {"fp64": total}
    assert pc.flops("fp64", prm) == {"fp64": inner, "fp32": total - inner}
    assert pc.flops("band", prm) == {"fp64": mid, "df64": total - mid}
    # an FP64 plan without a shell (rc64 >= rc) counts every pair on the FP64 pipe
    assert pc.flops("fp64", dict(prm, rc64=0.05)) == {"fp64": total}


def test_stage_model_band():
    prm = {"Mt": 16, "P": 8, "n_fft_in": 7, "n_fft_out": 4, "rc": 0.1, "rc64": 0.1}
    m = bench.stage_model("band", prm, 1000, 6, {"fp64": 1.0, "df64": 2.0})
    f = bench.stage_model("fp64", prm, 1000, 6, {"fp64": 1.0, "fp32": 2.0})
    assert set(m["real"][1]) == {"fp64", "df64"} and set(m["fft"][1]) == {"df64"}
    # the band changes only the real-space pipes: the Fourier part is the FP64 plan's
    for st in ("spread", "fft", "scale", "ifft", "gather"):
        assert m[st] == f[st]


def test_stage_roofline_path_fraction():
    peaks = {"hbm_gbs": 1000.0, "fp64_tflops": 1.0, "fp32_tflops": 64.0, "df64_tflops": 8.0}
    model = {"a": (1e9, {}),                      # 1 ms of HBM
             "b": (1e6, {"fp64": 2e9}),          # 2 ms of FP64
             "c": (1e6, {"fp64": 1e9, "fp32": 64e9})}  # 1 + 1 ms on two pipes
    st, path = bench.stage_roofline(model, {"a": 2.0, "b": 2.0, "c": 4.0}, peaks, 8.0)
    by = {s["stage"]: s for s in st}
    assert by["a"]["bound"] == "hbm" and math.isclose(by["a"]["frac"], 0.5)
    assert by["b"]["bound"].startswith("alu") and math.isclose(by["b"]["frac"], 1.0)
    assert math.isclose(by["c"]["roofline_ms"], 2.0) and math.isclose(by["c"]["frac"], 0.5)
    assert math.isclose(path, (1 + 2 + 2) / 8.0)


def test_stage_model_pipes():
    prm = {"Mt": 16, "P": 8, "n_fft_in": 7, "n_fft_out": 4, "rc": 0.1, "rc64": 0.05}
    m = bench.stage_model("fp64", prm, 1000, 6, {"fp64": 1.0, "fp32": 2.0})
    assert set(m["spread"][1]) == {"df64"} and set(m["real"][1]) == {"fp64", "fp32"}
    m = bench.stage_model("plain", prm, 1000, 6, {"fp64": 1.0})
    assert set(m["fft"][1]) == {"fp64"}
    mx = bench.stage_model("mixed", prm, 1000, 6, {"fp32": 1.0})
    # FP32 grids move half the bytes of FP64 ones
    assert mx["fft"][0] * 2 == m["fft"][0] and mx["scale"][0] * 2 == m["scale"][0]
