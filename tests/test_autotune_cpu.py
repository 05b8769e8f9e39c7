"""The autotuner's host logic without a GPU: bucket arithmetic, the JSON cache's round trip, and
which descriptor fields `apply` fills (native tile and split, emulated kernel class; modular
problems and fields the caller set are left alone)."""
from __future__ import annotations

import os
import tempfile

import pytest

from paper_1609_00076_gb300 import autotune, gbdgemm


def test_buckets():
    # output bucket: floor(log2(sqrt(m n))); k bucket: floor(log2(k)); degenerate sizes go to 0
    assert autotune.bucket_of(32, 32) == 5
    assert autotune.bucket_of(2048, 2048) == 11
    assert autotune.bucket_of(32, 2048) == 8  # sqrt(2^16) = 2^8
    assert autotune.bucket_of(63, 64) == 5 and autotune.bucket_of(64, 64) == 6
    assert autotune.bucket_of(0, 0) == 0 and autotune.bucket_of(1, 1) == 0
    assert autotune.kbucket_of(1) == 0 and autotune.kbucket_of(1023) == 9 and autotune.kbucket_of(1024) == 10
    assert autotune.kbucket_of(0) == 0


@pytest.fixture
def tuner():
    gbdgemm.load()  # save() records the library version (built in-tree if missing)
    return autotune.Autotuner(cache_path=os.path.join(tempfile.mkdtemp(), "sub", "tune.json"))


def test_untuned_lookups_are_the_library_defaults(tuner):
    assert tuner.tile_for(100, 100) == 0
    assert tuner.ksplit_for(100, 100, 2000) == 1
    assert tuner.emulated_class_for(1000, 1000, 1000) == 0


def test_cache_round_trip(tuner):
    tuner.table["9"] = {"tile": 64, "ms": {"32": 2.0, "64": 1.0}}
    tuner.split_table["6_11"] = {"ksplit": 8, "ms": {"1": 4.0, "8": 1.0}}
    tuner.emu_table["10_10"] = {"tile": 256, "ms": {"128": 2.0, "256": 1.0}}
    tuner.save()
    again = autotune.Autotuner(cache_path=tuner.cache_path)
    assert again.table == tuner.table and again.split_table == tuner.split_table
    assert again.emu_table == tuner.emu_table
    assert again.tile_for(512, 512) == 64 and again.tile_for(2048, 2048) == 0
    assert again.ksplit_for(64, 64, 2048) == 8 and again.ksplit_for(64, 64, 1024) == 1
    assert again.emulated_class_for(1024, 1024, 1024) == 256


def test_a_damaged_cache_reads_as_empty(tuner):
    os.makedirs(os.path.dirname(tuner.cache_path), exist_ok=True)
    with open(tuner.cache_path, "w") as f:
        f.write("{not json")
    t = autotune.Autotuner(cache_path=tuner.cache_path)
    assert t.table == {} and t.split_table == {} and t.emu_table == {}


def test_apply_fills_only_unset_fields_of_native_and_emulated_problems(tuner):
    tuner.table["9"] = {"tile": 64}
    tuner.split_table["9_11"] = {"ksplit": 4}
    tuner.emu_table["9_11"] = {"tile": 256}
    nat = dict(mode=gbdgemm.GBD_MODE_NATIVE, m=512, n=512, k=2048, tile=0, ksplit=0)
    nat_set = dict(mode=gbdgemm.GBD_MODE_NATIVE, m=512, n=512, k=2048, tile=32, ksplit=2)
    emu = dict(mode=gbdgemm.GBD_MODE_EMULATED, m=512, n=512, k=2048, tile=0)
    mod = dict(mode=gbdgemm.GBD_MODE_MODULAR, m=512, n=512, k=2048, tile=0)
    out = tuner.apply([nat, nat_set, emu, mod])
    assert out[0]["tile"] == 64 and out[0]["ksplit"] == 4
    assert out[1]["tile"] == 32 and out[1]["ksplit"] == 2
    assert out[2]["tile"] == 256 and "ksplit" not in out[2]
    assert out[3]["tile"] == 0  # modular problems keep the library's own choice
