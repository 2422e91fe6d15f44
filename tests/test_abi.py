"""The C ABI library loads and exports every entry point of include/*.h (CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2204_07485_gb300", "libbigmeans.so")


def _ensure_built():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(bm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    _ensure_built()
    lib = ctypes.CDLL(LIB)
    declared = _declared()
    assert "bm_create" in declared and "bm_fit_chunk" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    assert sorted(bm.EXPORTED) == _declared()


def test_invalid_shapes_rejected_before_any_device_work():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    bad = [dict(m=10, n=2, k=3, s=20), dict(m=10, n=2, k=11, s=10),
           dict(m=10, n=0, k=1, s=5), dict(m=10, n=2, k=0, s=5),
           dict(m=2**31, n=2, k=2, s=5), dict(m=10, n=2, k=2, s=5, kpp_trials=0),
           dict(m=10, n=2, k=2, s=5, init=7), dict(m=10, n=2, k=2, s=5, empty=5)]
    for kw in bad:
        cfg = bm.bm_config_default(**kw)
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_create(cfg, 0x1000)
        assert e.value.status == bm.BM_EINVAL
    with pytest.raises(bm.BigMeansError) as e:
        bm.bm_draw_chunk(10, 11, 0, 0, 0x1000)
    assert e.value.status == bm.BM_EINVAL


def test_status_strings():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    assert bm.bm_status_string(0) == "ok"
    assert bm.bm_status_string(4) == "device wait timed out"
    assert bm.bm_status_string(99) == "unknown status"


def test_config_defaults_follow_the_paper():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    cfg = bm.bm_config_default()
    assert cfg.max_iter == 300 and cfg.tol == 1e-4 and cfg.kpp_trials == 3
    assert cfg.graphs == 1
    assert cfg.init == bm.BM_INIT_KMEANSPP and cfg.empty == bm.BM_EMPTY_DEGENERATE


def test_server_entry_points_validate_without_a_device():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    cfg = bm.bm_server_config(0, 0, 1)
    sv = bm._vp()
    assert bm._lib.bm_server_create(bm.ctypes.byref(cfg), bm.ctypes.byref(sv)) == bm.BM_EINVAL
    assert bm._lib.bm_server_destroy(None) == bm.BM_OK
    assert bm._lib.bm_submit(None, None, None) == bm.BM_EINVAL
    assert bm._lib.bm_wait(None, 1, 0.0, None) == bm.BM_EINVAL
    assert bm._lib.bm_server_stats_get(None, None) == bm.BM_EINVAL


def test_selftest_rejects_out_of_range_limits_without_a_device():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    assert bm.bm_selftest_wait_timeout(0) == bm.BM_EINVAL
    assert bm.bm_selftest_wait_timeout(5000) == bm.BM_EINVAL


def test_group_entry_points_validate_without_a_device():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    ok = dict(P=0x1000, s=100, n=4, k=3, C=0x2000, mask=0x3000)
    bad = [dict(ok, s=2), dict(ok, n=0), dict(ok, k=0), dict(ok, P=None), dict(ok, C=None),
           dict(ok, mask=None)]
    for q in bad:
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_group_create([q])
        assert e.value.status == bm.BM_EINVAL
    for q in (dict(ok, k=129, s=1000), dict(ok, n=513)):
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_group_create([q])
        assert e.value.status == bm.BM_EUNSUPPORTED
    with pytest.raises(bm.BigMeansError) as e:
        bm.bm_group_create([ok], max_iter=-1)
    assert e.value.status == bm.BM_EINVAL
    out = bm._vp()
    assert bm._lib.bm_group_create(None, 1, 300, 1e-4, 1, None, bm.ctypes.byref(out)) == bm.BM_EINVAL
    assert bm._lib.bm_group_run(None, None, None) == bm.BM_EINVAL
    assert bm._lib.bm_group_destroy(None) == bm.BM_OK


def test_binding_keeps_borrowed_objects_until_the_handle_ends():
    # the library borrows the memory behind the pointers it is given; the
    # binding keeps the owning objects referenced until destroy / job end
    _ensure_built()
    import gc
    import weakref
    import paper_2204_07485_gb300 as bm

    class Owner:
        pass

    x = Owner()
    ref = weakref.ref(x)
    bm._hold(("ctx", 0xABC), x)
    del x
    gc.collect()
    assert ref() is not None
    bm._release(("ctx", 0xABC))
    gc.collect()
    assert ref() is None
    # a job that ends (its callback ran) before its submit registered it is
    # not held afterwards, and leaves nothing behind
    y = Owner()
    ref = weakref.ref(y)
    bm._release(("job", 7, 1), ended=True)
    bm._hold(("job", 7, 1), y)
    del y
    gc.collect()
    assert ref() is None
    assert ("job", 7, 1) not in bm._held and ("job", 7, 1) not in bm._held_ended
    # a job released normally after being held
    z = Owner()
    ref = weakref.ref(z)
    bm._hold(("job", 7, 2), z)
    del z
    bm._release(("job", 7, 2), ended=True)
    gc.collect()
    assert ref() is None and ("job", 7, 2) not in bm._held_ended


def test_fit_host_validates_without_a_device():
    _ensure_built()
    import numpy as np
    import paper_2204_07485_gb300 as bm
    X = np.zeros((10, 2), np.float32)
    cfg = bm.bm_config_default(m=10, n=2, k=2, s=5)
    with pytest.raises(bm.BigMeansError) as e:
        bm.bm_fit_host(cfg, None, 1)
    assert e.value.status == bm.BM_EINVAL
    with pytest.raises(bm.BigMeansError) as e:
        bm.bm_fit_host(cfg, X, -1)
    assert e.value.status == bm.BM_EINVAL
    for kw in (dict(k=6), dict(s=11), dict(n=0)):
        bad = bm.bm_config_default(**dict(dict(m=10, n=2, k=2, s=5), **kw))
        with pytest.raises(bm.BigMeansError) as e:
            bm.bm_fit_host(bad, X, 1)
        assert e.value.status == bm.BM_EINVAL


def test_binding_struct_layouts_match_the_header(tmp_path):
    # every ctypes structure of the binding has the size and field offsets of
    # the C struct it mirrors, as a C compiler lays the header out
    import shutil
    import subprocess
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [(bm.bm_config, "bm_config"), (bm.bm_fit_report, "bm_fit_report"),
             (bm.bm_server_config, "bm_server_config"), (bm.bm_job_result, "bm_job_result"),
             (bm.bm_job, "bm_job"), (bm.bm_server_stats_t, "bm_server_stats"),
             (bm.bm_group_problem, "bm_group_problem"), (bm.bm_group_result, "bm_group_result")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bigmeans.h"',
             'int main(void) {']
    expect = []
    for cls, cname in pairs:
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
            expect.append(getattr(cls, fname).offset)
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                           text=True).stdout.split()]
    assert got == expect


def test_binding_constants_match_the_header(tmp_path):
    # every BM_* integer the binding defines has the header's value
    import shutil
    import subprocess
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    header = open(os.path.join(ROOT, "include", "bigmeans.h")).read()
    names = sorted(n for n in dir(bm) if n.startswith("BM_") and isinstance(getattr(bm, n), int)
                   and re.search(r"\b%s\b" % n, header))
    assert len(names) >= 10
    lines = ['#include <stdio.h>', '#include "bigmeans.h"', 'int main(void) {']
    lines += ['  printf("%%lld\\n", (long long)(%s));' % n for n in names]
    lines += ['  return 0;', '}']
    src = tmp_path / "consts.c"
    exe = tmp_path / "consts"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                           text=True).stdout.split()]
    assert dict(zip(names, got)) == {n: getattr(bm, n) for n in names}


def test_binding_argument_counts_match_the_header():
    _ensure_built()
    import paper_2204_07485_gb300 as bm
    src = open(os.path.join(ROOT, "include", "bigmeans.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"\b(?:bm_status|void|const char\s*\*|int32_t|int64_t|uint64_t|size_t)\s+"
                       r"(bm_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S)
    assert sorted(d[0] for d in decls) == _declared()
    for name, params in decls:
        p = params.strip()
        n = 0 if p in ("", "void") else p.count(",") + 1
        argtypes = getattr(bm._lib, name).argtypes
        assert argtypes is not None and len(argtypes) == n, name
