"""The oracle and the C-ABI library's host code under AddressSanitizer and
UndefinedBehaviorSanitizer (CPU; the stand-in for a device memory checker on
the host side).

Builds liboracle_san.so (g++ -fsanitize=address,undefined) and libnrc_san.so
(the host code of every translation unit compiled and linked with the same
sanitizers; the compilers run without the sanitizer runtimes), then runs the whole `-m "not gpu"` suite in a child process with
libasan and libubsan preloaded, NRC_ORACLE_SANITIZE=1 and NRC_LIB_VARIANT=san,
stopping at the first sanitizer report.  Leak checking is off (the Python
interpreter itself keeps allocations until exit).
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    out = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return out if os.path.isabs(out) and os.path.exists(out) else None


def _env():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc's sanitizer runtimes are not installed")
    env = dict(os.environ)
    env.update({"LD_PRELOAD": f"{asan} {ubsan}", "ASAN_OPTIONS": "detect_leaks=0:abort_on_error=1",
                "UBSAN_OPTIONS": "halt_on_error=1:print_stacktrace=1", "NRC_LIB_VARIANT": "san",
                "NRC_ORACLE_SANITIZE": "1", "PYTHONPATH": ROOT})
    return env


@pytest.fixture(scope="module")
def env():
    e = _env()
    # the sanitized libraries are built without the runtimes preloaded: the
    # compilers themselves are not meant to run under them (nvcc has crashed so)
    build_env = {k: v for k, v in e.items() if k not in ("LD_PRELOAD", "ASAN_OPTIONS", "UBSAN_OPTIONS")}
    code = ("from paper_2106_12372_gb300 import build; build.build(); from oracle import oracle; oracle.build()")
    subprocess.run([sys.executable, "-c", code], env=build_env, cwd=ROOT, check=True, timeout=900)
    return e


def test_sanitized_libraries_are_the_ones_loaded(env):
    code = ("from paper_2106_12372_gb300 import nrc; from oracle import oracle as O; nrc.lib(); O.lib(); "
            "m = open('/proc/self/maps').read(); "
            "print(all(k in m for k in ('libasan', 'libnrc_san.so', 'liboracle_san.so')))")
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().endswith("True"), out.stdout


def test_cpu_suite_is_clean_under_asan_and_ubsan(env):
    cmd = [sys.executable, "-m", "pytest", "tests", "-m", "not gpu", "-q", "-x", "-p", "no:cacheprovider",
           "--ignore=tests/test_sanitizers.py"]
    out = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=1500)
    tail = (out.stdout + out.stderr)[-4000:]
    assert out.returncode == 0, tail
    assert "AddressSanitizer" not in tail and "runtime error" not in tail, tail
