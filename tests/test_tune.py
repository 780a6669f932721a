"""Host logic of the autotuner: size buckets and the cache file (CPU)."""
import json

import pytest

pytest.importorskip("torch")

import paper_1710_10096_gb300 as sff
from paper_1710_10096_gb300 import tune


@pytest.fixture(scope="module", autouse=True)
def built():
    sff.build()


def test_size_buckets():
    assert tune.size_bucket(1242, 375) == "1280x384"
    assert tune.size_bucket(1280, 384) == "1280x384"
    assert tune.size_bucket(1281, 385) == "1344x416"
    assert tune.size_bucket(8, 8) == "64x32"


def test_cache_round_trip_skips_unsupported_entries(tmp_path):
    saved = dict(tune._CACHE)
    try:
        tune._CACHE.clear()
        params = tuple(sff.default_params().as_dict().values())
        good = {"variants": [sff.VARIANT_SPACE[1], (1, 0, 32, 16, 4), (0, 0, 0, 0, 0), (1, 4, 16, 8, 0)],
                "pair": 1, "alt": 5, "pdl": 0, "fuse": 8, "tma": 0}
        tune._CACHE[("1280x384", params)] = good
        path = tmp_path / "tuning.json"
        tune.save_cache(str(path))
        data = json.loads(path.read_text())
        pk = ",".join(map(str, params))
        ok = data["1280x384|" + pk]
        data["640x192|" + pk] = dict(ok, variants=[[3, 0, 32, 8, 0]] * 4)  # not a supported variant
        data["512x160|" + pk] = dict(ok, variants=[[4, 4, 16, 8, 0]] * 4)  # region beyond 1024 threads
        data["448x160|" + pk] = dict(ok, pair=2)  # not a schedule
        data["384x160|" + pk] = dict(ok, alt=16)  # not a scale bit mask
        data["320x160|" + pk] = dict(ok, pdl=-1)  # not a scale bit mask
        data["320x128|" + pk] = dict(ok, variants=ok["variants"][:3] + [[4, 4, 8, 8, 0]], fuse=8)  # no fused form
        data["320x96|" + pk] = dict(ok, fuse=1)  # scale 0 is never fused
        data["320x64|" + pk] = dict(ok, pdl=8)  # fused and dependent launch on one scale
        data["320x32|" + pk] = dict(ok, variants=[[2, 0, 32, 8, 0]] + ok["variants"][1:], tma=1)  # no TMA form
        data["288x32|" + pk] = dict(ok, tma=2)  # not 0 / 1
        data["256x96|" + pk] = [1, 0, 32, 8]  # an old (one variant) format
        data["128x64|" + pk] = [[1, 0, 32, 8, 0]] * 4  # an old (list of variants) format
        path.write_text(json.dumps(data))
        tune._CACHE.clear()
        assert tune.load_cache(str(path)) == 1
        e = tune._CACHE[("1280x384", params)]
        assert e == {"variants": [tuple(v) for v in good["variants"]], "pair": 1, "alt": 5, "pdl": 0, "fuse": 8,
                     "tma": 0}
        t = tune._tuning_of(e)
        assert t.scale_variants() == [tuple(v) for v in good["variants"]]
        assert (t.pair_fields, t.alternate_order, t.pdl, t.fuse) == (1, 5, 0, 8)
        assert tune.load_cache(str(tmp_path / "missing.json")) == 0
    finally:
        tune._CACHE.clear()
        tune._CACHE.update(saved)


def test_variant_space_matches_the_library():
    # every listed variant is accepted at every scale; nearby settings that
    # the library does not instantiate are refused
    for v in sff.VARIANT_SPACE:
        l, c, tx, ty, mb = v
        t = sff.make_tuning(l, tx, ty, c, [v] * 3, min_ctas=mb)
        assert t.scale_variants() == [v] * 4
    for bad in [(4, 4, 16, 8, 0), (2, 4, 32, 8, 0), (4, 1, 64, 8, 0), (2, 1, 64, 16, 0), (1, 2, 32, 8, 0),
                (3, 0, 32, 8, 0), (1, 0, 32, 16, 5), (2, 0, 32, 16, 4), (1, 1, 32, 16, 4)]:
        assert bad not in sff.VARIANT_SPACE
        with pytest.raises(sff.SffError):
            sff.make_tuning(bad[0], bad[2], bad[3], bad[1], min_ctas=bad[4])
        with pytest.raises(sff.SffError):
            sff.make_tuning(1, 32, 16, 0, [bad])
    assert len(sff.VARIANT_SPACE) == 45
    for bad_sched in [dict(group_mb=-1), dict(pair_fields=2), dict(alternate_order=16), dict(alternate_order=-1),
                      dict(pdl=16), dict(features_form=3), dict(features_form=-1)]:
        with pytest.raises(sff.SffError):
            sff.make_tuning(1, 32, 16, 0, None, **bad_sched)


def test_fused_space_matches_the_library():
    # every fused variant is accepted at every coarse scale with its fuse bit
    for v in sff.FUSED_SPACE:
        assert v in sff.VARIANT_SPACE
        t = sff.make_tuning(1, 32, 16, 0, [v] * 3, fuse=14)
        assert t.fuse == 14 and t.scale_variants()[1:] == [v] * 3
    # refused: scale 0 fused, a fused scale with a variant that has no fused
    # form, fuse sharing a bit with pdl or alternate_order, bits beyond the
    # scales
    fv = sff.FUSED_SPACE[0]
    no_fused = [v for v in sff.VARIANT_SPACE if v not in sff.FUSED_SPACE]
    assert (1, 0, 64, 16, 0) in no_fused and (4, 4, 8, 8, 0) in no_fused
    for kw in [dict(coarse=[fv] * 3, fuse=1), dict(coarse=[(1, 0, 64, 16, 0)] * 3, fuse=2), dict(coarse=[(4, 4, 8, 8, 0)] * 3, fuse=8),
               dict(coarse=[(1, 0, 32, 16, 3)] * 3, fuse=4),
               dict(coarse=[fv] * 3, fuse=2, pdl=2), dict(coarse=[fv] * 3, fuse=6, alternate_order=4),
               dict(coarse=[fv] * 3, fuse=16), dict(coarse=[fv] * 3, fuse=-2)]:
        with pytest.raises(sff.SffError):
            sff.make_tuning(1, 32, 16, 0, **kw)
    # the other bits of the same scales stay free
    t = sff.make_tuning(1, 32, 16, 0, [fv] * 3, fuse=6, pdl=9, alternate_order=1)
    assert (t.fuse, t.pdl, t.alternate_order) == (6, 9, 1)
    # derived coarse variants (all-zero entries) always have a fused form
    assert sff.make_tuning(1, 32, 16, 0, None, fuse=14).fuse == 14
    assert sff.make_tuning(1, 32, 16, 0, [fv, (0,) * 5, fv], fuse=4).fuse == 4


def test_tma_space_matches_the_library():
    # every TMA variant is accepted as the scale-0 variant with tma = 1;
    # other scale-0 variants and values other than 0 / 1 are refused
    for v in sff.TMA_SPACE:
        assert v in sff.VARIANT_SPACE
        t = sff.make_tuning(v[0], v[2], v[3], v[1], None, min_ctas=v[4], tma=1)
        assert t.tma == 1 and t.scale_variants()[0] == v
    for v in [(1, 0, 64, 16, 0), (2, 0, 32, 8, 0), (1, 1, 32, 8, 0), (1, 0, 32, 16, 4)]:
        assert v not in sff.TMA_SPACE
        with pytest.raises(sff.SffError):
            sff.make_tuning(v[0], v[2], v[3], v[1], None, min_ctas=v[4], tma=1)
    with pytest.raises(sff.SffError):
        sff.make_tuning(1, 32, 16, 0, None, tma=2)
