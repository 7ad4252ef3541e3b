"""Host-side arithmetic of the benchmark: the algorithmic byte counts behind
the roofline figures follow the library's own octave geometry, and the clock
sampler reads nvidia-smi's CSV as documented."""
import ctypes
import os

import pytest

import bench
import paper_2605_17869_gb300 as pkg
from paper_2605_17869_gb300 import _abi


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_17869_gb300 import build
    build.build()


def _geometry(H, W, upsample):
    p = _abi.SiftParams()
    _abi.load().sift_params_default(ctypes.byref(p))
    p.upsample, p.upsample_max_px = int(upsample), 0
    return pkg.sift_octave_geometry(p, H, W)[2]


@pytest.mark.parametrize("shapes,up", [([(750, 1000)] * 6, True), ([(480, 640), (97, 211), (1200, 1600)], False),
                                       ([(16, 16), (31, 47)], True)])
def test_algorithmic_bytes_follow_the_library_geometry(shapes, up):
    """Level blurs: S + 2 per octave, 8 B per octave pixel each (one read, one
    write), plus 4 B per pixel for the decimating first blur of octaves above 0.
    Base: input read (4 B/px) and level 0 written. Extrema: the S + 3 levels read
    and S bits of bitmap per octave pixel."""
    S = 3
    blur = px = base = ext = 0
    for (h, w) in shapes:
        geo = _geometry(h, w, up)
        base += 4 * h * w + 4 * geo[0][0] * geo[0][1]
        for o, (H, W) in enumerate(geo):
            blur += 8 * H * W * (S + 2) + (4 * H * W if o else 0)
            px += H * W * (S + 2)
            ext += 4 * (S + 3) * H * W + S * H * W // 8
    assert bench._alg_blur_bytes(shapes, up) == (blur, px)
    assert bench._alg_class_bytes(shapes, up) == {"base": base, "extrema": ext}


def test_timed_workload_blur_bytes_per_launch():
    """6 x 1000x750, magnified: octaves 2000x1500 down to 31x23 (7 octaves, 35
    level-blur launches); 983,852,160 algorithmic bytes per step, 28.1 MB per
    launch."""
    b, _ = bench._alg_blur_bytes([(750, 1000)] * 6, True)
    assert b == 983_852_160
    assert len(_geometry(750, 1000, True)) == 7


class _Proc:
    def terminate(self):
        pass

    def wait(self):
        return 0


def test_clock_sampler_parses_the_csv(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("0, 1965, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 1980, 2070, 910.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1995, 2070, 920.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
        f.write("0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c.proc, c.f = _Proc(), open(os.devnull, "w")
    got = c.stop()
    assert got == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_sampler_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop() is None


@pytest.mark.parametrize("S,sigma0", [(3, 1.6), (4, 1.6), (2, 1.3)])
def test_level_radii_follow_the_oracle_taps(S, sigma0):
    """The dual roofline's FP32 count uses the level blurs' radii: they must be
    the oracle's ceil(4 kappa_i) for the increments kappa_i of §3.2."""
    from oracle import sift_oracle as so
    p = so.Params()
    p.n_scales, p.sigma0 = S, sigma0
    assert bench._level_radii(S, sigma0) == [so.gaussian_taps(k)[0] for k in so.increment_sigmas(p)]


def test_blur_flops_count_every_level_of_every_octave():
    """4 (2R + 1) FLOP per octave pixel per level blur (two passes of 2R + 1
    FMAs), summed over the library's octaves."""
    shapes = [(480, 640), (97, 211)]
    radii = bench._level_radii()
    want = sum(H * W * sum(4 * (2 * r + 1) for r in radii)
               for h, w in shapes for (H, W) in _geometry(h, w, False))
    assert bench._alg_blur_flops(shapes, False) == want


def test_default_tuning_is_recognised():
    d = ('{"blur_tile_rows": [[32, 32, 32, 32, 32]], "blur_ctas_per_sm": [0], '
         '"extrema_ctas_per_sm": 0, "orientation_ctas_per_sm": 0, "descriptor_ctas_per_sm": 0, '
         '"compaction_ctas_per_sm": 0}')
    assert bench._is_default_tuning(d)
    assert bench._is_default_tuning('{"blur_tile_rows": [32, 32, 32, 32, 32]}')
    assert not bench._is_default_tuning(d.replace('"extrema_ctas_per_sm": 0', '"extrema_ctas_per_sm": 4'))
    assert not bench._is_default_tuning(d.replace("[[32, 32, 32, 32, 32]]",
                                                  "[[32, 32, 32, 32, 32], [32, 64, 32, 32, 32]]"))
    assert not bench._is_default_tuning(d.replace('"blur_ctas_per_sm": [0]', '"blur_ctas_per_sm": [0, 3]'))
    assert bench._is_default_tuning(d[:-1] + ', "batch_lanes": 2}')
    assert not bench._is_default_tuning(d[:-1] + ', "batch_lanes": 1}')


class _FakeCuda:
    """Stand-in for torch.cuda: events read a clock that each step advances,
    so that the timing helpers can be checked without a device."""

    def __init__(self, clock):
        self.clock = clock

    def synchronize(self):
        pass

    def Event(self, enable_timing=False):
        clock = self.clock

        class Ev:
            def record(self, stream=None):
                self.t = clock[0]

            def synchronize(self):
                pass

            def elapsed_time(self, other):
                return other.t - self.t

        return Ev()


class _FakeTorch:
    def __init__(self, clock):
        self.cuda = _FakeCuda(clock)


def test_queued_steps_time_exactly_the_queued_steps():
    clock = [0.0]
    calls = []

    def step():  # each step costs 2 ms of "device" time
        clock[0] += 2.0
        calls.append(1)

    ms, wall = bench.queued_steps(_FakeTorch(clock), step, 7, 3, None)
    assert len(calls) == 10 and ms == 14.0 and wall >= 0.0


def test_best_queued_ms_takes_the_fastest_run():
    clock = [0.0]
    costs = iter([5.0] * 4 + [9.0] * 3 + [5.0] * 4 + [2.0] * 3 + [5.0] * 4 + [4.0] * 3)

    def step():  # warm-up steps cost 5 ms; the three timed runs 9, 2 and 4 ms per step
        clock[0] += next(costs)

    assert bench.best_queued_ms(_FakeTorch(clock), step, 9, 4, None) == 2.0
