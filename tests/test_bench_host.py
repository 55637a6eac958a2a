"""bench.py's host logic (no GPU): the hash that keys recorded ncu counters to
the kernel code, and the scaling of the recorded DRAM traffic to a launch."""
import importlib.util
import json
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tree(tmp_path, name):
    """A copy of the kernel sources under tmp_path/name, laid out like the repo."""
    root = tmp_path / name
    csrc = root / "paper_0811_3448_gb300" / "csrc"
    csrc.parent.mkdir(parents=True)
    src = os.path.join(ROOT, "paper_0811_3448_gb300", "csrc")
    shutil.copytree(src, csrc, ignore=shutil.ignore_patterns("__pycache__"))
    (root / "profiles").mkdir()
    return root, csrc


def test_source_hash_ignores_comments_not_code(tmp_path):
    b = _bench()
    base, _ = _tree(tmp_path, "base")
    commented, c2 = _tree(tmp_path, "commented")
    changed, c3 = _tree(tmp_path, "changed")
    k = c2 / "kernels.cuh"
    k.write_text(k.read_text().replace("namespace binar {", "// a note\nnamespace binar {  /* x */", 1))
    k = c3 / "kernels.cuh"
    text = k.read_text()
    assert "kLookbackWindow = 8" in text
    k.write_text(text.replace("kLookbackWindow = 8", "kLookbackWindow = 4", 1))
    hashes = {}
    for name, root in (("base", base), ("commented", commented), ("changed", changed)):
        b.ROOT = str(root)
        hashes[name] = b.kernel_source_hash()
    assert hashes["base"] == hashes["commented"]
    assert hashes["base"] != hashes["changed"]
    # code outside the kernel files (the string levels, the C ABI) does not count
    other, c4 = _tree(tmp_path, "other")
    k = c4 / "strings.cu"
    k.write_text(k.read_text() + "\nstatic int unrelated_code = 1;\n")
    b.ROOT = str(other)
    assert b.kernel_source_hash() == hashes["base"]


def test_recorded_traffic_matches_widths_and_scales_per_record(tmp_path):
    b = _bench()
    root, _ = _tree(tmp_path, "t")
    b.ROOT = str(root)
    rec = {"source_hash": b.kernel_source_hash(),
           "kernels": {"partition[0]": {"key_bytes": 4, "val_bytes": 4, "measured_keys": 1000,
                                        "dram_bytes_read": 7000, "dram_bytes_write": 8000}}}
    (root / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert b.recorded_traffic("partition[0]", 4, 4, 1000) == 15000
    assert b.recorded_traffic("partition[0]", 4, 4, 8000) == 120000
    assert b.recorded_traffic("partition[0]", 8, 4, 1000) is None     # other key width
    assert b.recorded_traffic("partition[0]", 4, 0, 1000) is None     # keys alone
    assert b.recorded_traffic("finish[3]", 4, 4, 1000) is None
    rec["source_hash"] = "0" * 16                                      # kernels changed since
    (root / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert b.recorded_traffic("partition[0]", 4, 4, 1000) is None
