"""Pins the oracle's binar sort to the paper's worked example.

The fixture tests/golden/worked_example.txt transcribes every partition
configuration that the paper prints for the nybble array [B 4 0 0 7 A C E]
("Illustration of the Algorithm": first pass, the passes on both sub-arrays at
the second bit, the per-bit summary for bits 1-2, and the final array).
"""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def _nyb(tokens):
    return [int(t, 16) for t in tokens]


def _parse():
    states, levels, final, inp = [], {}, None, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("input"):
                inp = _nyb(line.split()[1:])
            elif line.startswith("state"):
                head, body = line.split("|")
                _, pos, lower, upper = head.split()
                groups = [g.split() for g in body.strip()[1:-1].split("][")]
                assert len(groups) == 3
                states.append((int(pos), int(lower), int(upper), [_nyb(g) for g in groups]))
            elif line.startswith("level"):
                head, body = line.split("|")
                levels[int(head.split()[1])] = [_nyb(g.split()) for g in body.split(";")]
            elif line.startswith("final"):
                final = _nyb(line.split()[1:])
    return inp, states, levels, final


def _render(row, n):
    pos, lower, upper, lo, hi = (int(v) for v in row[:5])
    arr = [int(v) >> 4 for v in row[5:5 + n]]
    return (pos, lower, upper,
            [arr[lower:lo], arr[lo:hi + 1], arr[hi + 1:upper + 1]])


def test_worked_example_states_and_result():
    inp, states, levels, final = _parse()
    keys = (np.array(inp, dtype=np.uint8) << 4).astype(np.uint8)
    trace = oracle.binar_sort_trace(keys, w=4)
    n = len(inp)
    rendered = [_render(r, n) for r in trace]
    printed_ranges = {(p, lo, up) for p, lo, up, _ in states}
    got = [s for s in rendered if (s[0], s[1], s[2]) in printed_ranges]
    assert got == states
    assert [int(k) >> 4 for k in keys] == final


def test_worked_example_level_membership():
    inp, states, levels, final = _parse()
    keys = (np.array(inp, dtype=np.uint8) << 4).astype(np.uint8)
    trace = oracle.binar_sort_trace(keys.copy(), w=4)
    n = len(inp)
    # array after the last placement at bit 0, and after the last at bit 1
    for level, groups in levels.items():
        rows = [r for r in trace if r[0] == level - 1]
        arr = [int(v) >> 4 for v in rows[-1][5:5 + n]]
        flat = [x for g in groups for x in g]
        assert sorted(arr) == sorted(flat)
        at = 0
        for g in groups:
            assert sorted(arr[at:at + len(g)]) == sorted(g)
            at += len(g)


def test_worked_example_visits_bound():
    # the time analysis: every element is visited at most once per bit
    keys = (np.array([0xB, 4, 0, 0, 7, 0xA, 0xC, 0xE], dtype=np.uint8) << 4).astype(np.uint8)
    visits = oracle.binar_sort(keys, w=4)
    assert 0 < visits <= 4 * 8
