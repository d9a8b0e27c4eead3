"""Autotuner choices kept across processes (paper_1202_6163_gb300.tuning): the
JSON file's layout, the size classes, and which choices a later process sets,
with the library's timing and setter replaced by fakes (no GPU)."""
import json

import pytest

from paper_1202_6163_gb300 import pf, tuning

KEY = "GB300-test|152 SMs|sm_103"


def test_size_class_is_ceil_log2():
    # brute force: the smallest c with 2^c >= P
    for P in list(range(1, 5000)) + [(1 << 20) - 1, 1 << 20, (1 << 20) + 1, (1 << 25) - 3, 1 << 31, (1 << 40) + 7]:
        c = 0
        while (1 << c) < P and c < tuning.N_CLASSES - 1:
            c += 1
        assert tuning.size_class(P) == c, P
    with pytest.raises(ValueError):
        tuning.size_class(0)


def test_record_then_load_sets_only_this_devices_choices(tmp_path, monkeypatch):
    path = str(tmp_path / "tiles.json")
    tuning.record(path, KEY, pf.PF_SYSTEMATIC, 1 << 20, 4096)
    tuning.record(path, KEY, pf.PF_SYSTEMATIC, 5000, 1024)
    tuning.record(path, KEY, pf.PF_MULTINOMIAL, 300000, 6144)
    tuning.record(path, KEY, pf.PF_SYSTEMATIC, (1 << 20) - 5, 8192)  # same class as 2^20: replaces it
    tuning.record(path, "another GPU|132 SMs|sm_90", pf.PF_STRATIFIED, 1 << 20, 3072)
    with open(path) as f:
        data = json.load(f)
    assert data == {"version": 1, "devices": {
        KEY: {"systematic": {"20": 8192, "13": 1024}, "multinomial": {"19": 6144}},
        "another GPU|132 SMs|sm_90": {"stratified": {"20": 3072}}}}

    calls = []
    monkeypatch.setattr(pf, "pf_set_min_tile", lambda kind, P, t: calls.append((kind, P, t)))
    assert tuning.load(path, key=KEY) == 3
    assert sorted(calls) == sorted([(pf.PF_SYSTEMATIC, 1 << 20, 8192), (pf.PF_SYSTEMATIC, 1 << 13, 1024),
                                    (pf.PF_MULTINOMIAL, 1 << 19, 6144)])
    # each P passed back lies in the class it was stored under
    for kind, P, _ in calls:
        assert str(tuning.size_class(P)) in data["devices"][KEY][tuning.KIND_NAMES[kind]]
    calls.clear()
    assert tuning.load(path, key="unknown|1 SMs|sm_00") == 0
    assert tuning.load(str(tmp_path / "missing.json"), key=KEY) == 0
    assert calls == []


def test_tune_and_record_stores_the_autotuners_pick(tmp_path, monkeypatch):
    path = str(tmp_path / "tiles.json")
    seen = []

    def fake_autotune(kind, logw, P, ancestors, reps=20, stream=None):
        seen.append((kind, logw, P, ancestors, reps, stream))
        return 3072, 17.5

    monkeypatch.setattr(pf, "pf_autotune", fake_autotune)
    assert tuning.tune_and_record(path, pf.PF_STRATIFIED, "lw", 70000, "anc", reps=7, key=KEY) == (3072, 17.5)
    assert seen == [(pf.PF_STRATIFIED, "lw", 70000, "anc", 7, None)]
    assert tuning.read(path)["devices"] == {KEY: {"stratified": {"17": 3072}}}


@pytest.mark.parametrize("content", [
    "[]",
    '{"version": 2, "devices": {}}',
    '{"version": 1}',
    '{"version": 1, "devices": {"k": {"metropolis": {"20": 4096}}}}',
    '{"version": 1, "devices": {"k": {"systematic": {"x": 4096}}}}',
    '{"version": 1, "devices": {"k": {"systematic": {"32": 4096}}}}',
    '{"version": 1, "devices": {"k": {"systematic": {"20": -1}}}}',
    '{"version": 1, "devices": {"k": {"systematic": {"20": 40.5}}}}',
    '{"version": 1, "devices": {"k": 3}}',
])
def test_malformed_files_are_rejected(tmp_path, content):
    path = tmp_path / "tiles.json"
    path.write_text(content)
    with pytest.raises(ValueError):
        tuning.read(str(path))


def test_metropolis_has_no_tile_choice(tmp_path):
    with pytest.raises(ValueError):
        tuning.record(str(tmp_path / "tiles.json"), KEY, pf.PF_METROPOLIS, 1 << 20, 4096)
    assert not (tmp_path / "tiles.json").exists()
