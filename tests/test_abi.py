"""The C ABI library builds, loads and exports every entry point include/pdv.h
declares; the Python binding's ctypes layouts match the C header. No compute
call is made here (this runs without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2012_00963_gb300 import build as B
from paper_2012_00963_gb300 import pdv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pdv_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_functions():
    assert declared_functions() == sorted(pdv.ABI_FUNCTIONS)


@pytest.mark.parametrize("debug", [False, True], ids=["release", "debug"])
def test_library_builds_and_exports_every_symbol(debug):
    path = B.build(debug=debug)
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (pdv_[a-z0-9_]+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    L = C.CDLL(path)
    for name in declared_functions():
        assert getattr(L, name) is not None


def test_ctypes_layouts_match_the_header(tmp_path):
    """sizeof/offsetof of every public struct, from a C program compiled
    against include/pdv.h, equal the binding's ctypes layouts."""
    structs = {
        "pdv_cloud_desc": pdv.pdv_cloud_desc, "pdv_probe": pdv.pdv_probe,
        "pdv_counters": pdv.pdv_counters, "pdv_request": pdv.pdv_request,
        "pdv_tuning": pdv.pdv_tuning, "pdv_cloud_info": pdv.pdv_cloud_info,
        "pdv_stats": pdv.pdv_stats, "pdv_allocator": pdv.pdv_allocator,
        "pdv_ss_set": pdv.pdv_ss_set, "pdv_peak_opts": pdv.pdv_peak_opts,
        "pdv_peak": pdv.pdv_peak, "pdv_debug_info": pdv.pdv_debug_info,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdv.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (sname, sname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (sname, f, sname, f))
    lines.append('printf("pdv_packet_record %zu\\n", sizeof(pdv_packet_record));')
    for f in pdv.TRACE_DTYPE.names:
        lines.append('printf("pdv_trace_vertex.%s %%zu\\n", offsetof(pdv_trace_vertex, %s));' % (f, f))
    lines.append('printf("pdv_trace_vertex %zu\\n", sizeof(pdv_trace_vertex));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for sname, cls in structs.items():
        assert int(got[sname]) == C.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (sname, f)]) == getattr(cls, f).offset, (sname, f)
    assert int(got["pdv_packet_record"]) == pdv.PACKET_DTYPE.itemsize
    assert int(got["pdv_trace_vertex"]) == pdv.TRACE_DTYPE.itemsize
    for f in pdv.TRACE_DTYPE.names:
        assert int(got["pdv_trace_vertex." + f]) == pdv.TRACE_DTYPE.fields[f][1], f
    assert C.sizeof(pdv.pdv_peak) == pdv.PEAK_DTYPE.itemsize
    assert C.sizeof(pdv.pdv_ss_set) == pdv.SS_SET_DTYPE.itemsize


def test_status_codes_and_error_path_without_gpu():
    """Without a usable device the context call fails with a CUDA status and a
    message instead of crashing; nothing falls back to the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pdv.PdvError) as e:
        pdv.pdv_ctx_create(0)
    assert e.value.status in (pdv.PDV_ECUDA, pdv.PDV_EINVAL)
    assert pdv.last_error()
