"""Host side of the native request loop (no GPU): the job record's layout
matches include/pi.h, the slot charge is as documented, and bad server
arguments are rejected before any device call."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2406_16091_gb300 import binding as B
from paper_2406_16091_gb300 import build as pibuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIELDS = [f[0] for f in B.PiJob._fields_]


def test_job_record_layout_matches_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pi.h"', "int main(void) {",
             '  printf("size %zu\\n", sizeof(pi_job));']
    lines += [f'  printf("{f} %zu\\n", offsetof(pi_job, {f}));' for f in FIELDS]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(B.PiJob)
    for f in FIELDS:
        assert int(out[f]) == getattr(B.PiJob, f).offset, f


def test_slot_charge():
    pibuild.build()
    assert B.pi_server_slot_bytes(65536) == 65536 * 144 + (1 << 20)
    from paper_2406_16091_gb300.serving import slot_bytes

    assert slot_bytes(65536, 65536) == B.pi_server_slot_bytes(65536)


@pytest.mark.parametrize("caps,init,maxs", [([], [], 8), ([1024, 1024], [0, 0], 8), ([1024], [0], 0),
                                            ([0], [0], 8), ([1024], [-1], 8), ([1 << 31], [0], 8)])
def test_server_rejects_bad_arguments(caps, init, maxs):
    pibuild.build()
    if not caps:
        st = B.load().pi_server_create(0, None, None, 8, 0, ctypes.byref(ctypes.c_void_p()))
        assert st == B.PI_ERR_INVALID_ARG
        return
    with pytest.raises(B.PiError) as e:
        B.pi_server_create(caps, init, maxs, 0)
    assert e.value.status == B.PI_ERR_INVALID_ARG


def test_server_calls_reject_null():
    pibuild.build()
    L = B.load()
    assert L.pi_server_run(None, None, 0, None) == B.PI_ERR_INVALID_ARG
    assert L.pi_server_info(None, None, None, None, None) == B.PI_ERR_INVALID_ARG
    assert L.pi_server_destroy(None) == B.PI_OK
