"""The host thread pool that builds a batch call's work list (spl_host_pool.h),
compiled with g++ and run on the CPU: every chunk runs exactly once, over
repeated runs, concurrent runs from four host threads and a forked child."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_pool_runs_every_chunk_once(tmp_path):
    exe = tmp_path / "host_pool_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I",
                    os.path.join(ROOT, "paper_2509_20500_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_pool_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
