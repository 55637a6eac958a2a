"""Shows that the oracle pins catch plausible mistakes.

Each case copies oracle/binar_oracle.c, plants one mistake (a dropped term, a
wrong sign or bound, a reversed loop), builds the copy with gcc into a
temporary directory, and runs a subset of the pins against it: at least one
pin must fail.  Nothing here touches a GPU.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import MAP_FLOAT, MAP_SIGNED
from paper_0811_3448_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "binar_oracle.c")

MUTANTS = {
    "loop_bound": ("while (below < above) {", "while (below + 1 < above) {"),
    "dropped_exchange": ("above--;\n                exchange(r, below, above);", "above--;"),
    "float_negatives": ("if (negative) b = !b;", "if (0) b = !b;"),
    "signed_bit": ("if (map == MAP_SIGNED) {\n        if (pos == 0) b = !b;",
                   "if (map == MAP_SIGNED) {\n        if (pos == 1) b = !b;"),
    "radix_direction": ("for (int pos = w - 1; pos >= 0; pos--) {",
                        "for (int pos = 0; pos < w; pos++) {"),
    "digit_weight": ("d = 2 * d + b;\n        }\n        digit[i] = d;",
                     "d = d + b;\n        }\n        digit[i] = d;"),
    "upper_recursion": ("(pending){below, upper, pos + 1}", "(pending){below, upper, pos + 2}"),
    "parallel_group_bits": ("g = 2 * g + key_bit(keys + i * kb, kb, map, p);", "g = 2 * g;"),
    "parallel_start_bit": ("jobs[g].pos = b;", "jobs[g].pos = b + 1;"),
    "parallel_group_bounds": ("jobs[g].upper = count[g + 1] - 1;", "jobs[g].upper = count[g + 1] - 2;"),
    "string_prefix_rule": ("if (la != lb) return la < lb ? -1 : 1;", "if (la != lb) return 0;"),
    "string_byte_order": ("if (sa[i] != sb[i]) return sa[i] < sb[i] ? -1 : 1;",
                          "if (sa[i] != sb[i]) return sa[i] > sb[i] ? -1 : 1;"),
    "string_stability": ("compare_strings(bytes, offsets, order[j], order[i]) < 0",
                         "compare_strings(bytes, offsets, order[j], order[i]) <= 0"),
}


def _pins_pass(lib) -> bool:
    """Runs a compact subset of the pins against `lib`; False if any fails."""
    saved = oracle._lib
    oracle._lib = lib
    try:
        # worked-example result and exhaustive 4-nybble arrays
        length, rows = 4, 16 ** 4
        digits = np.indices((16,) * length).reshape(length, -1).T.astype(np.uint8)
        keys = (digits << 4).astype(np.uint8).reshape(-1)
        expect = np.sort(keys.reshape(rows, length), axis=1).reshape(-1)
        oracle.binar_sort(keys, w=4, offsets=np.arange(rows + 1, dtype=np.int64) * length)
        if not np.array_equal(keys, expect):
            return False
        # signed and float order against numpy
        k = inputs.config3_i64(3000)
        e = np.sort(k)
        oracle.binar_sort(k, key_map=MAP_SIGNED)
        if not np.array_equal(k, e):
            return False
        f = inputs.config3_f32(3000)
        oracle.binar_sort(f, key_map=MAP_FLOAT)
        if not np.all(np.diff(f[np.isfinite(f)].astype(np.float64)) >= 0):
            return False
        # stable radix against a stable argsort
        k = inputs.config2_keys(3000, np.uint32, "distinct8")
        v = inputs.index_payload(3000)
        order = np.argsort(k, kind="stable")
        k2, v2 = k.copy(), v.copy()
        oracle.stable_radix(k2, v2)
        if not np.array_equal(v2, v[order]):
            return False
        # one partition pass against a stable argsort of the digit
        k = inputs.uniform_keys(3000, np.uint32, np.random.Generator(np.random.PCG64(1)))
        ko, vo, offs = oracle.partition_pass(k, v, pos=4, k=8)
        digit = (k >> np.uint32(20)) & np.uint32(255)
        if not np.array_equal(vo, v[np.argsort(digit, kind="stable")]):
            return False
        # the parallel variant against np.sort, payload pointing at its key
        k = inputs.uniform_keys(5000, np.uint32, np.random.Generator(np.random.PCG64(2)))
        v = inputs.index_payload(5000)
        k2, v2 = k.copy(), v.copy()
        oracle.binar_sort_parallel(k2, v2, log2_groups=4)
        if not (np.array_equal(k2, np.sort(k)) and np.array_equal(k[v2], k2)):
            return False
        # strings: prefixes, equal strings in input order
        data = np.frombuffer(b"ab" + b"a" + b"ab" + b"b" + b"" + b"a", dtype=np.uint8).copy()
        off = np.array([0, 2, 3, 5, 6, 6, 7], dtype=np.int64)
        if list(oracle.sort_strings(data, off)) != [4, 1, 5, 0, 2, 3]:
            return False
        return True
    finally:
        oracle._lib = saved


def test_unmutated_oracle_passes_the_subset():
    assert _pins_pass(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(path)])
    lib = oracle.configure(ctypes.CDLL(str(so)))
    assert not _pins_pass(lib), f"mutant {name} survived the pins"
