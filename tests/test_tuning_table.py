"""The tuned launch table compiled into the library (csrc/polaris_tuning.h, written by
paper_1412_1256_gb300/tune.py): well-formed entries, a lossless writer/reader pair, and
agreement with the measurement record beside it."""
import json
import os

from paper_1412_1256_gb300 import tune


def test_table_entries_are_valid():
    entries = tune.parse_header(open(tune.HEADER).read())
    seen = set()
    for (logn, bits, mb, c1, c2) in entries:
        assert 4 <= logn <= 20 and bits in (1, 2, 4, 8)
        assert mb >= 0 and c1 in (0, 1, 2, 3) and c2 in (0, 1, 2)
        assert (logn, bits) not in seen
        seen.add((logn, bits))


def test_writer_and_reader_agree():
    entries = [(17, 2, 64, 0, 1), (10, 8, 0, 1, 0)]
    assert sorted(tune.parse_header(tune.render_header(entries))) == sorted(entries)
    assert tune.parse_header(tune.render_header([])) == []


def test_table_matches_its_measurement_record():
    entries = tune.parse_header(open(tune.HEADER).read())
    if not os.path.exists(tune.RECORD):
        assert entries == []
        return
    rec = json.load(open(tune.RECORD))
    chosen = {tuple(int(x) for x in k.split(",")): tuple(v["chosen"]) for k, v in rec["results"].items()}
    for (logn, bits, mb, c1, c2) in entries:
        assert chosen[(logn, bits)] == (mb, c1, c2)
    for (logn, bits), ch in chosen.items():
        if ch != (0, 0, 0):
            assert (logn, bits) + ch in entries
        r = rec["results"][f"{logn},{bits}"]
        # an entry leaves the built-in choice only for a gain above the record's threshold
        if ch != (0, 0, 0):
            assert r["all"][",".join(map(str, ch))] > r["builtin"] * (1 + rec["min_gain"])
