"""Stand-ins for a memory/race checker, which is not available on this
pool: two checking builds of the same sources, each run in a child process
on jobs that reach every kernel family and the host-side runtime
(tests/checking_build_jobs.py), with results compared against the product
build's.

  * guards: device index guards compiled in (BM_DEBUG_GUARDS).  An access
    outside its buffer is skipped and reported as BM_EGUARD through the
    launch's status word; nothing traps.  Every job must succeed with the
    product build's results bit for bit.
  * asan: the host code built with AddressSanitizer and UndefinedBehavior-
    Sanitizer (runtimes preloaded into the child).  Any report fails the
    test; results must equal the product build's.

The CPU test runs the host-only entry points under the sanitizers here; the
GPU tests run the whole job list on the device.
"""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
JOBS = os.path.join(ROOT, "tests", "checking_build_jobs.py")


def _builder():
    spec = importlib.util.spec_from_file_location(
        "_bm_build_variants", os.path.join(ROOT, "paper_2204_07485_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _sanitizer_env(lib):
    def rt(name):
        r = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True)
        return r.stdout.strip()
    env = dict(os.environ, BM_LIBRARY=lib)
    env["LD_PRELOAD"] = rt("libasan.so")
    # CUDA maps memory in the range ASan keeps as its shadow gap; leaks of the
    # interpreter itself are not this library's
    env["ASAN_OPTIONS"] = "protect_shadow_gap=0:detect_leaks=0:halt_on_error=1"
    env["UBSAN_OPTIONS"] = "halt_on_error=1:print_stacktrace=1"
    return env


def _run(mode, env, timeout=900):
    r = subprocess.run([sys.executable, JOBS, mode], capture_output=True, text=True,
                       env=env, timeout=timeout, cwd=ROOT)
    return r


def _check_clean(r):
    bad = [ln for ln in r.stderr.splitlines()
           if "AddressSanitizer" in ln or "runtime error:" in ln or "LeakSanitizer" in ln]
    assert r.returncode == 0 and not bad, (r.returncode, bad[:5], r.stderr[-2000:])


def test_host_entry_points_under_asan_ubsan():
    lib = _builder().build(variant="asan")
    r = _run("host", _sanitizer_env(lib))
    _check_clean(r)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["create_bad"] == 1 and res["status"][8].startswith("device index guard")


@pytest.mark.gpu
def test_device_index_guards_find_nothing():
    b = _builder()
    ref = _run("gpu", dict(os.environ))
    assert ref.returncode == 0, ref.stderr[-2000:]
    lib = b.build(variant="guards")
    r = _run("gpu", dict(os.environ, BM_LIBRARY=lib))
    assert r.returncode == 0, r.stderr[-3000:]   # a tripped guard raises BM_EGUARD
    assert json.loads(r.stdout.strip().splitlines()[-1]) == \
        json.loads(ref.stdout.strip().splitlines()[-1])


@pytest.mark.gpu
def test_host_code_under_asan_ubsan_on_the_device():
    b = _builder()
    ref = _run("gpu", dict(os.environ))
    assert ref.returncode == 0, ref.stderr[-2000:]
    lib = b.build(variant="asan")
    r = _run("gpu", _sanitizer_env(lib))
    _check_clean(r)
    assert json.loads(r.stdout.strip().splitlines()[-1]) == \
        json.loads(ref.stdout.strip().splitlines()[-1])
