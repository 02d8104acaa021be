"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/rtgb.h; the binding's struct layouts match the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtgb.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^RT_API\s+[\w\s\*]+?\b(rt_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1203_2941_gb300.builder import build
    path = build()
    return ctypes.CDLL(path), path


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rt_\w+)", out))
    assert set(names) <= exported
    from paper_1203_2941_gb300 import rtgb
    assert set(rtgb.EXPORTS) == set(names)


def test_calls_without_gpu_fail_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L, _ = lib
    L.rt_version.restype = ctypes.c_char_p
    assert b"rtgb" in L.rt_version()
    h = ctypes.c_void_p()
    assert L.rt_ctx_create(0, ctypes.byref(h)) != 0
    L.rt_last_error.restype = ctypes.c_char_p
    assert len(L.rt_last_error()) > 0


def test_struct_layouts_match_header():
    from paper_1203_2941_gb300 import rtgb as R
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "rtgb.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(rt_source), sizeof(rt_transport_params),
         sizeof(rt_transport_out), sizeof(rt_camera), sizeof(rt_model), sizeof(rt_event),
         sizeof(rt_pah_event), sizeof(rt_traj));
  printf("%zu %zu %zu\n", offsetof(rt_transport_params, march_min_active),
         offsetof(rt_transport_out, stats), offsetof(rt_model, out));
  printf("%zu %zu %zu %zu\n", sizeof(rt_pc_camera), offsetof(rt_transport_params, pc_cams),
         offsetof(rt_transport_out, pc_img), offsetof(rt_transport_params, record_nu_mask));
  return 0;
}
'''
    tmp = os.path.join(ROOT, "oracle", "_build")
    os.makedirs(tmp, exist_ok=True)
    c = os.path.join(tmp, "layout.c")
    exe = os.path.join(tmp, "layout")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    got = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    want = [ctypes.sizeof(R.rt_source), ctypes.sizeof(R.rt_transport_params),
            ctypes.sizeof(R.rt_transport_out), ctypes.sizeof(R.rt_camera), ctypes.sizeof(R.rt_model),
            R.EVENT_DTYPE.itemsize, R.PAH_DTYPE.itemsize, R.TRAJ_DTYPE.itemsize,
            R.rt_transport_params.march_min_active.offset, R.rt_transport_out.stats.offset,
            R.rt_model.out.offset,
            ctypes.sizeof(R.rt_pc_camera), R.rt_transport_params.pc_cams.offset,
            R.rt_transport_out.pc_img.offset, R.rt_transport_params.record_nu_mask.offset]
    assert [int(v) for v in got] == want
