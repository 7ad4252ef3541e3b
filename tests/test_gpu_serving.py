"""Serving (continuous batching) and autotuning on the GPU.

Each served result must be bit-identical to the same image extracted alone:
requests are batched with whatever else is in flight, and batching never
changes an image's arithmetic. Autotuned tile shapes change only the work
distribution, so tuned and default runs must also agree bit for bit."""
import time

import numpy as np
import pytest

from workloads import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_17869_gb300 as pkg  # noqa: E402


def _same(a, b):
    if a.count != b.count:
        return False
    return all(torch.equal(x, y) for x, y in ((a.x, b.x), (a.y, b.y), (a.sigma, b.sigma),
                                             (a.angle, b.angle), (a.response, b.response),
                                             (a.octave, b.octave), (a.layer, b.layer),
                                             (a.desc, b.desc)))


def test_served_results_equal_singleton_runs():
    shapes = [(480, 640), (1080, 1920), (300, 411), (480, 640), (720, 1280), (97, 211)] * 3
    imgs = [torch.from_numpy(synth.make_image(synth.rng_for(40, i), *s)).cuda()
            for i, s in enumerate(shapes)]
    ref_ex = pkg.Extractor(max_kpts=4096)
    refs = [ref_ex.extract(im) for im in imgs]
    ex = pkg.Extractor(max_kpts=4096)
    srv = pkg.Server(ex, budget_bytes=2 << 30, max_slots=8)
    tickets = [srv.submit(im) for im in imgs]       # arrive while others run
    lat = []
    for t, r in zip(tickets, refs):
        f, ms, st = srv.result(t)
        assert st in (pkg.SIFT_OK, pkg.SIFT_W_TRUNCATED)
        assert _same(f, r)
        lat.append(ms)
        srv.release(t)
    assert all(v > 0 for v in lat)
    srv.close()


def test_admitted_requests_overlap_on_the_device_and_match_singletons():
    """Continuous batching: requests that arrive while others are on the GPU
    are admitted into steps on the other lanes, and those steps run on the
    device at the same time (their CUDA-event intervals intersect); each result
    is still bit-identical to the image extracted alone."""
    shapes = [(1080, 1920), (480, 640), (720, 1280), (1080, 1920), (600, 800), (1080, 1920)] * 4
    imgs = [torch.from_numpy(synth.make_image(synth.rng_for(42, i), *s)).cuda()
            for i, s in enumerate(shapes)]
    ref_ex = pkg.Extractor(max_kpts=2048)
    refs = [ref_ex.extract(im) for im in imgs]
    torch.cuda.synchronize()
    ex = pkg.Extractor(max_kpts=2048)
    srv = pkg.Server(ex, budget_bytes=4 << 30, max_slots=8)
    tickets = []
    for im in imgs:                              # each arrives while earlier ones run
        tickets.append(srv.submit(im))
        time.sleep(2e-4)
    for t, r in zip(tickets, refs):
        f, _, st = srv.result(t)
        assert st in (pkg.SIFT_OK, pkg.SIFT_W_TRUNCATED)
        assert _same(f, r)
        srv.release(t)
    steps = srv.steps()
    assert sum(n for _, n, _, _ in steps) == len(imgs)
    assert all(t1 > t0 for _, _, t0, t1 in steps)
    overlaps = [(a, b) for i, a in enumerate(steps) for b in steps[i + 1:]
                if a[0] != b[0] and a[2] < b[3] and b[2] < a[3]]
    print(f"{len(steps)} steps on lanes {sorted(set(s[0] for s in steps))}, "
          f"{len(overlaps)} overlapping pairs on different lanes")
    assert overlaps, steps
    srv.close()


def test_poll_and_release_protocol():
    ex = pkg.Extractor(max_kpts=1024)
    srv = pkg.Server(ex, budget_bytes=1 << 30, max_slots=4)
    img = torch.from_numpy(synth.single_vga(3)).cuda()
    t = srv.submit(img)
    f = None
    for _ in range(20000):
        f = srv.poll(t)
        if f is not None:
            break
    if f is None:
        f, _, _ = srv.result(t)
    assert f.count > 0
    srv.release(t)
    with pytest.raises(pkg.SiftError) as e:
        srv.release(t)
    assert e.value.status == pkg.SIFT_E_NOTFOUND
    srv.close()


def test_budget_rejects_oversized_request():
    ex = pkg.Extractor(max_kpts=1024)
    srv = pkg.Server(ex, budget_bytes=8 << 20, max_slots=4)
    big = torch.zeros((2160, 3840), device="cuda")
    with pytest.raises(pkg.SiftError) as e:
        srv.submit(big)
    assert e.value.status == pkg.SIFT_E_BUDGET
    srv.close()


def test_autotuned_tiles_bit_identical():
    img = torch.from_numpy(synth.make_image(synth.rng_for(41, 0), 700, 900)).cuda()
    a = pkg.Extractor()
    fa = a.extract(img)
    b = pkg.Extractor()
    js = b.autotune(700, 900)
    assert "blur_tile_rows" in js
    fb = b.extract(img)
    assert _same(fa, fb)
    for rows in ("[32, 32, 32, 32, 32]", "[64, 64, 64, 64, 64]", "[64, 32, 64, 32, 64]"):
        b.set_tuning('{"blur_tile_rows": %s}' % rows)
        assert _same(fa, b.extract(img))


def _batch_feats(ex, n):
    bufs = ex._buffers(n)
    counts = ex._counts[:n].tolist()
    return [pkg.Features(*(t.clone() for t in (f.x, f.y, f.sigma, f.angle, f.response, f.octave,
                                               f.layer, f.desc)), c)
            for f, c in ((b.view(c), c) for b, c in zip(bufs, counts))]


def test_tuning_json_round_trip_and_validation():
    ex = pkg.Extractor()
    js = ('{"blur_tile_rows": [[64, 32, 64, 32, 32], [32, 64, 32, 32, 32]], '
          '"blur_ctas_per_sm": [2, 3], "extrema_ctas_per_sm": 3, '
          '"orientation_ctas_per_sm": 5, "descriptor_ctas_per_sm": 4, '
          '"compaction_ctas_per_sm": 2, "batch_lanes": 1}')
    ex.set_tuning(js)
    assert ex.get_tuning() == js
    ex.set_tuning('{"blur_tile_rows": [32, 32, 32, 32, 64]}')  # flat list: octave 0 only
    assert ex.get_tuning().startswith('{"blur_tile_rows": [[32, 32, 32, 32, 64], '
                                      '[32, 64, 32, 32, 32]]')
    for bad in ('{"blur_tile_rows": [48, 32, 32, 32, 32]}', '{"blur_tile_rows": [32, 32]}',
                '{"extrema_ctas_per_sm": 65}', '{"extrema_ctas_per_sm": -1}', '{"grid": 1}',
                '{"descriptor_ctas_per_sm": 2.5}', '[]', '{"blur_ctas_per_sm": [1] } x',
                '{"batch_lanes": 5}', '{"batch_lanes": 0}'):
        with pytest.raises(pkg.SiftError):
            ex.set_tuning(bad)
    ex.close()


def test_batch_autotune_bit_identical_and_cached(tmp_path):
    shapes = [(480, 640), (1200, 1600), (300, 411), (720, 1280), (97, 211), (900, 700)]
    imgs = [torch.from_numpy(synth.make_image(synth.rng_for(42, i), *s, fractal_std=0.05)).cuda()
            for i, s in enumerate(shapes)]
    ref = pkg.Extractor().extract_batch(imgs)  # default tuning
    cache = str(tmp_path / "tuning.json")
    ex = pkg.Extractor()
    js, hit = ex.autotune_batch(imgs, cache=cache)
    assert not hit
    torch.cuda.synchronize()
    tuned = _batch_feats(ex, len(imgs))  # the autotuner leaves the chosen tuning's results
    assert all(_same(a, b) for a, b in zip(ref, tuned))
    assert all(_same(a, b) for a, b in zip(ref, ex.extract_batch(imgs)))
    ex.close()
    # A second handle finds the tuning in the cache, also for the batch reversed.
    ex2 = pkg.Extractor()
    js2, hit2 = ex2.autotune_batch(imgs[::-1], cache=cache)
    assert hit2 and js2 == js
    torch.cuda.synchronize()
    assert all(_same(a, b) for a, b in zip(ref[::-1], _batch_feats(ex2, len(imgs))))
    ex2.close()
    # Every corner of the search space gives the same bits.
    ex3 = pkg.Extractor()
    for t in ('{"blur_tile_rows": [[64, 64, 64, 64, 64], [64, 64, 64, 64, 64], '
              '[64, 64, 64, 64, 64]], "blur_ctas_per_sm": [1, 1, 1], "extrema_ctas_per_sm": 1, '
              '"orientation_ctas_per_sm": 1, "descriptor_ctas_per_sm": 1, '
              '"compaction_ctas_per_sm": 1, "batch_lanes": 1}',
              '{"blur_ctas_per_sm": [2, 3, 2, 1], "extrema_ctas_per_sm": 2, '
              '"orientation_ctas_per_sm": 4, "descriptor_ctas_per_sm": 3, '
              '"compaction_ctas_per_sm": 3, "batch_lanes": 2}',
              '{"batch_lanes": 1}'):
        ex3.set_tuning(t)
        assert all(_same(a, b) for a, b in zip(ref, ex3.extract_batch(imgs)))
    ex3.close()


def test_batch_lanes_bit_identical_with_pack_and_stats():
    """A batch in 2, 3 or 4 concurrent parts (batch_lanes) against the whole
    batch in one pass: the same features, the same packed download, the same
    per-image stats; the caller's stream sees every part without a
    device-wide synchronisation."""
    shapes = [(1200, 1600), (97, 211), (480, 640), (720, 1280), (300, 411)]
    imgs = [torch.from_numpy(synth.make_image(synth.rng_for(77, i), *s, fractal_std=0.05)).cuda()
            for i, s in enumerate(shapes)]
    one = pkg.Extractor()
    one.set_tuning('{"batch_lanes": 1}')
    assert '"batch_lanes": 2' in pkg.Extractor().get_tuning()
    side = torch.cuda.Stream()
    for lanes in (2, 3, 4):
        many = pkg.Extractor()
        many.set_tuning('{"batch_lanes": %d}' % lanes)
        for batch in (imgs, imgs[:2], imgs[1:4], imgs[:1], imgs[::-1]):
            fa = one.extract_batch(batch)
            with torch.cuda.stream(side):
                bufs, cnt = many.extract_batch_async(batch, side)
                counts = cnt.clone()
            side.synchronize()  # only the caller's stream: it must have joined every part
            fb = [b.view(c) for b, c in zip(bufs, counts.tolist())]
            assert len(fa) == len(fb)
            assert all(_same(a, b) for a, b in zip(fa, fb)), (lanes, len(batch))
            ca, pa = one.download()
            cb, pb = many.download(side)
            assert ca == cb == [f.count for f in fa]
            for a, b in zip(pa, pb):
                for k in a:
                    assert np.array_equal(a[k], b[k]), k
            sa, ra = one.stats(len(batch))
            sb, rb = many.stats(len(batch))
            assert sa == sb and ra == rb
            if len(batch) >= 2:  # every part launches its own graph
                assert many.launch_count() > one.launch_count()
        many.close()
    one.close()
