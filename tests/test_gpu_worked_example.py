"""The paper's worked example ("Illustration of the Algorithm") on the GPU.

The nybble array [B 4 0 0 7 A C E] is placed in the top 4 bits of uint32 keys.
One 8-bit partition pass at bit 0 groups the keys by their top byte, so the
paper's sub-arrays after its first and second bit are unions of adjacent digit
buckets.  Their membership must equal the printed summary as multisets (the
order inside a sub-array differs: the paper's exchange is unstable, the pass
is stable).  The full sorts must give the printed final array, and the pair
sort the stable order of the payloads.
"""
import numpy as np
import pytest

from gpu_util import expect_pairs, require_gpu, same_bits, to_dev, to_host
from paper_0811_3448_gb300 import binding
from test_oracle_worked_example import _parse

pytestmark = pytest.mark.gpu


def test_worked_example_sub_arrays_after_bits_1_and_2():
    require_gpu()
    inp, _, levels, final = _parse()
    keys = np.array(inp, dtype=np.uint32) << np.uint32(28)
    vals = np.arange(keys.shape[0], dtype=np.uint32)
    ko, vo, offs = binding.partition_pass(to_dev(keys), to_dev(vals), pos=0)
    ko, vo, offs = to_host(ko), to_host(vo), to_host(offs)
    assert offs[0] == 0 and offs[256] == keys.shape[0]
    for bits, groups in sorted(levels.items()):
        got = []
        for prefix in range(1 << bits):
            a, b = offs[prefix << (8 - bits)], offs[(prefix + 1) << (8 - bits)]
            if b > a:
                got.append(sorted(int(k) >> 28 for k in ko[a:b]))
        assert got == [sorted(g) for g in groups], bits
    # the pass moved every key with its payload
    assert np.array_equal(keys[vo], ko)


def test_worked_example_final_array():
    require_gpu()
    inp, _, _, final = _parse()
    keys = np.array(inp, dtype=np.uint32) << np.uint32(28)
    tk = to_dev(keys)
    binding.sort_keys(tk)
    assert [int(k) >> 28 for k in to_host(tk)] == final
    vals = np.arange(keys.shape[0], dtype=np.uint32)
    tk, tv = to_dev(keys), to_dev(vals)
    binding.sort_pairs(tk, tv)
    ek, ev = expect_pairs(keys, vals)
    assert same_bits(to_host(tk), ek) and same_bits(to_host(tv), ev)
    assert [int(k) >> 28 for k in ek] == final
