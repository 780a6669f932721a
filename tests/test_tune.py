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
        good = sff.TUNING_SPACE[0]
        tune._CACHE[("1280x384", params)] = good
        path = tmp_path / "tuning.json"
        tune.save_cache(str(path))
        data = json.loads(path.read_text())
        data["640x192|" + ",".join(map(str, params))] = [3, 32, 8]  # not a supported tuning
        path.write_text(json.dumps(data))
        tune._CACHE.clear()
        assert tune.load_cache(str(path)) == 1
        assert tune._CACHE == {("1280x384", params): tuple(good)}
        assert tune.load_cache(str(tmp_path / "missing.json")) == 0
    finally:
        tune._CACHE.clear()
        tune._CACHE.update(saved)
