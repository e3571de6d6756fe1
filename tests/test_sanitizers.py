"""AddressSanitizer + UndefinedBehaviorSanitizer runs on the CPU:

  * the FP64 oracle (plain C), driven through every entry point on a small
    ragged batch with all physics switches on (tests/c/oracle_sanitize.c);
  * the C ABI's host code (the whole library built with host-side
    sanitizers; the device code is unchanged), driven through every entry
    point's argument checks and no-device paths (tests/c/abi_sanitize.c).

Both abort on the first error; leak checking is off for the second, whose
process also holds the CUDA runtime's own allocations.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=all"]


def test_oracle_under_asan_ubsan(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    exe = tmp_path / "oracle_san"
    subprocess.run(["gcc", "-std=c11", "-O1", "-g", *SAN, "-Wno-unknown-pragmas",
                    os.path.join(ROOT, "oracle", "oracle.c"), os.path.join(ROOT, "tests", "c", "oracle_sanitize.c"),
                    "-o", str(exe), "-lm"], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr[-3000:]
    assert "oracle sanitized run" in r.stdout


def test_abi_host_code_under_asan_ubsan(tmp_path):
    from paper_2203_11043_gb300 import build
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not found")
    src = build.CSRC
    xc = [a for f in SAN for a in ("-Xcompiler", f)]
    procs, objs = [], []
    for f in build.SOURCES:
        o = str(tmp_path / (f + ".o"))
        objs.append(o)
        procs.append(subprocess.Popen([nvcc, *build.ARCH, "-O1", "-g", "-std=c++17", *xc, "-I", build.INCLUDE,
                                       "-I", src, "-c", os.path.join(src, f), "-o", o],
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for p in procs:
        out, _ = p.communicate()
        assert p.returncode == 0, out.decode()[-3000:]
    drv = str(tmp_path / "drv.o")
    subprocess.run(["gcc", "-std=c11", "-g", *SAN, "-I", build.INCLUDE, "-c",
                    os.path.join(ROOT, "tests", "c", "abi_sanitize.c"), "-o", drv], check=True, capture_output=True)
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    exe = str(tmp_path / "abi_san")
    subprocess.run(["g++", *SAN, drv, *objs, "-L", cuda_lib, "-lcudart_static", "-ldl", "-lpthread", "-lrt",
                    "-o", exe], check=True, capture_output=True)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stdout + r.stderr[-3000:]
    assert "ABI host code sanitized run: ok" in r.stdout
