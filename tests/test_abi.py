"""The C ABI library loads, exports every entry point declared in include/moss103.h, and
rejects invalid parameters before touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np

import pytest

from paper_2405_12520_b300 import build, moss, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "moss103.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\**\s*(ms_\w+)\s*\(", hdr, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("ms_create", "ms_load_network", "ms_add_vehicles", "ms_step", "ms_read_state",
              "ms_write_state", "ms_read_metrics", "ms_read_debug", "ms_last_error", "ms_destroy", "ms_sync"):
        assert f in names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = C.CDLL(moss.LIB_PATH)
    for f in _declared():
        assert hasattr(lib, f), f
    assert set(moss.SYMBOLS) <= set(_declared())


@pytest.mark.parametrize("bad", [dict(dt=0.0), dict(p_lc=1.5), dict(a_min=1.0), dict(v_max=0.0),
                                 dict(window=0)])
def test_create_rejects_invalid_params(bad):
    build.build()
    p = synth.default_params(**bad)
    with pytest.raises(moss.MossError) as e:
        moss.Sim(p)
    assert e.value.code == moss.MS_ERR_ARG


def test_create_rejects_bad_block():
    build.build()
    with pytest.raises(moss.MossError) as e:
        moss.Sim(synth.default_params(), block=100)
    assert e.value.code == moss.MS_ERR_ARG


def test_header_is_plain_c_and_links_from_c(tmp_path):
    """A C99 translation unit that includes the header and takes the address of every entry
    point compiles with gcc and links against the library (no C++ types or mangling)."""
    import subprocess
    build.build()
    names = _declared()
    src = tmp_path / "abi.c"
    src.write_text('#include "moss103.h"\n#include <stdio.h>\nint main(void) {\n  void *fns[] = {\n' +
                   "".join(f"    (void *){n},\n" for n in names) +
                   '  };\n  printf("%d\\n", (int)(sizeof fns / sizeof fns[0]));\n  return 0;\n}\n')
    exe = tmp_path / "abi"
    libdir = os.path.dirname(moss.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-l:" + os.path.basename(moss.LIB_PATH), "-Wl,-rpath," + libdir])
    assert exe.exists()


def test_export_buffers_bound_the_copy():
    """The binding hands the library the length of the smallest export buffer, and refuses
    buffers that are not contiguous 4-byte tensors (the library writes float32 / int32)."""
    import torch
    from paper_2405_12520_b300 import moss
    assert moss._export_capacity(torch.zeros(5), torch.zeros(3, dtype=torch.int32), None) == 3
    for bad in (torch.zeros(4, dtype=torch.float64), torch.zeros(8)[::2]):
        with pytest.raises(ValueError):
            moss._export_capacity(bad)
    with pytest.raises(ValueError):
        moss._export_capacity(None, None)


def test_binding_checks_input_lengths_before_the_library_reads_them():
    """Arrays the library reads a counted number of elements from are checked in the
    binding first (a mismatch raises before any call into the library, so no device or
    library state is needed here)."""
    import torch
    from paper_2405_12520_b300 import moss
    s = object.__new__(moss.Sim)          # the checks run before the library is used
    with pytest.raises(ValueError):
        s.set_lane_limits([1, 2], vmax=[3.0])
    with pytest.raises(ValueError):
        s.set_lane_limits([1, 2], closed=[1, 0, 1])
    with pytest.raises(ValueError):
        s.set_lane_links([1, 2], [0])
    with pytest.raises(ValueError):
        s.sample_trips([0, 1, 2], [1.0, 2.0], 2, 10, 60, 1)
    with pytest.raises(ValueError):
        s.sample_trips_radiation([0, 1], [1.0], 10, 60, 1)
    with pytest.raises(ValueError):
        s.set_lc_model(np.zeros(moss.MLP_NPARAM - 1, np.float32))
    x = torch.zeros((8, 16), dtype=torch.bfloat16)
    y = torch.zeros(8, dtype=torch.int32)
    n = torch.zeros(1, dtype=torch.int32)
    with pytest.raises(ValueError):
        s.set_lc_log(x, y)                                          # n missing
    with pytest.raises(ValueError):
        s.set_lc_log(x.float(), y, n)                               # not bf16
    with pytest.raises(ValueError):
        s.set_lc_log(torch.zeros((8, 15), dtype=torch.bfloat16), y, n)   # not 16 inputs
