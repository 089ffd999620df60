"""The launch-configuration cache file (SPL_TUNE_CACHE) read back on the host:
each line is "padded-N pass-kind SMs threads state-level blocks-per-SM
[columns-per-thread]" (8 columns when the last field is absent); lookups find
the entry of their batch kind and nothing else, and a file that breaks off
mid-line keeps the entries before it.  No GPU: without a device
the library's SM count is 1, which the keys below use."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = (
    "import json\n"
    "from paper_2509_20500_gb300 import spl\n"
    "print(json.dumps([spl.batch_tune_lookup(2000), spl.batch_tune_lookup(2000, spl.SPL_PASS_STRUCTURED),\n"
    "                  spl.batch_tune_lookup(700), spl.batch_tune_lookup(9000)]))\n")


def _lookup(path):
    env = dict(os.environ, SPL_TUNE_CACHE=str(path), PYTHONPATH=ROOT, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", CODE], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    import json
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_cache_file_entries_are_found_by_kind(tmp_path):
    # padded lengths: 2000 -> 2048, 700 -> 768 (multiples of 256 for 8 columns per thread)
    f = tmp_path / "tune.txt"
    f.write_text("2048 0 1 256 2 2\n2048 1 1 256 1 3 8\n768 0 1 512 0 1 4\n")
    dense, structured, small, big = _lookup(f)
    assert dense == [256, 2, 2, 8]          # a line without the column count: 8
    assert structured == [256, 1, 3, 8]
    assert small == [512, 0, 1, 4]
    assert big is None                      # nothing cached for that size


def test_cache_file_broken_off_keeps_earlier_entries(tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("2048 0 1 256 2 2 4\n768 0 1 2")   # the second line breaks off
    dense, structured, small, big = _lookup(f)
    assert dense == [256, 2, 2, 4] and structured is None and small is None


def test_missing_cache_file_means_nothing_cached(tmp_path):
    dense, structured, small, big = _lookup(tmp_path / "absent.txt")
    assert dense is None and structured is None and small is None and big is None
