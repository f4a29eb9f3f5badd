"""CPU checks of the tuning table (host logic of libflood's flood_tuning_* entry points).

The table maps a workload bucket (SM count, log2 points, log2 landmarks, m)
to the grid cell factor and the heavy-group shell threshold; lookups take
the nearest bucket among entries for the current device's SM count, else the
defaults. Entries round-trip through the text file the autotuner writes.
"""
import pytest
import torch

from paper_2509_22432_b300 import tune
from paper_2509_22432_b300._lib import FloodError


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count if torch.cuda.is_available() else 1


@pytest.fixture(autouse=True)
def empty_table():
    tune.clear()
    yield
    tune.clear()


def test_defaults_without_entries():
    assert tune.lookup(1_000_000, 2000, 10) == {"cell_factor": 0.5, "heavy_shells": 9, "tuned": False}


def test_nearest_bucket_and_other_gpus():
    sms = _sms()
    tune.set_entry(tune.bucket(1_000_000, 2000, 10, sms), 0.7, 10)
    tune.set_entry(tune.bucket(5_000_000, 10_000, 12, sms), 1.0, 8)
    tune.set_entry(tune.bucket(5_000_000, 10_000, 12, sms + 1), 0.35, 12)      # another GPU: never used here
    assert tune.lookup(1_000_000, 2000, 10)["cell_factor"] == pytest.approx(0.7)
    assert tune.lookup(1_100_000, 2100, 10)["heavy_shells"] == 10               # same bucket (log2 rounds)
    got = tune.lookup(4_000_000, 9000, 12)
    assert got["tuned"] and got["heavy_shells"] == 8 and got["cell_factor"] == pytest.approx(1.0)
    assert tune.bucket(1_000_000, 2000, 10, sms) == (sms, 20, 11, 10)


def test_replace_and_file_round_trip(tmp_path):
    sms = _sms()
    key = tune.bucket(200_000, 4000, 8, sms)
    tune.set_entry(key, 0.5, 9)
    tune.set_entry(key, 0.7, 11)                                               # same bucket: replaced
    tune.set_entry(tune.bucket(2_000, 40, 8, sms), 0.35, 7)
    assert len(tune.entries()) == 2
    path = str(tmp_path / "tune.txt")
    tune.save(path)
    text = open(path).read()
    assert text.startswith("#") and f"{sms} 18 12 8 0.7 11" in text
    tune.clear()
    assert tune.lookup(200_000, 4000, 8)["tuned"] is False
    assert tune.load(path) == 2
    assert tune.lookup(200_000, 4000, 8) == {"cell_factor": pytest.approx(0.7), "heavy_shells": 11, "tuned": True}


def test_bad_entries_and_files_are_rejected(tmp_path):
    with pytest.raises(FloodError):
        tune.set_entry((1, 20, 11, 10), 0.0, 9)          # cell factor must be positive
    with pytest.raises(FloodError):
        tune.set_entry((1, 20, 11, 10), 0.5, 64)         # at most 63 shell classes
    bad = tmp_path / "bad.txt"
    bad.write_text("# header\n1 20 11 10 0.5 9\nnot an entry\n")
    with pytest.raises(FloodError):
        tune.load(str(bad))
    assert len(tune.entries()) == 1                      # the line before the bad one stays
    with pytest.raises(FloodError):
        tune.load(str(tmp_path / "missing.txt"))


def test_choice_keeps_the_defaults_unless_a_candidate_is_clearly_faster():
    from paper_2509_22432_b300 import tune
    d = tune.DEFAULTS
    # a near-tie (0.16 %): the defaults stay
    assert tune.choose({(0.7, 7): 1.6367, d: 1.6393, (1.0, 12): 2.0}) == (d, 1.6393)
    # clearly faster (10 %): the candidate wins
    assert tune.choose({(0.7, 10): 1.80, d: 2.00}) == ((0.7, 10), 1.80)
    # just past the margin
    assert tune.choose({(0.35, 8): 1.0, d: 1.0 * (1.0 + tune.KEEP_DEFAULTS_WITHIN) * 1.001}) == ((0.35, 8), 1.0)
    # defaults not measured: the fastest
    assert tune.choose({(0.35, 6): 3.0, (1.0, 12): 2.5}) == ((1.0, 12), 2.5)
    # defaults fastest
    assert tune.choose({(0.35, 6): 3.0, d: 2.0}) == (d, 2.0)
