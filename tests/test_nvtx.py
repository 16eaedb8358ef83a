"""NVTX ranges of the library: every API entry that reaches the device pushes
a range named after the call; inside it the spectrum call has ranges for the
transport launch and the normalisation, and the serving thread one per launch
and per normalisation. Each test runs a child process with a counting NVTX
injection library (tests/nvtx_count.c, built here with gcc) named by
NVTX_INJECTION64_PATH, and checks the counts and that every push was popped
on its own thread."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def injection(tmp_path_factory):
    out = tmp_path_factory.mktemp("nvtx") / "libnvtx_count.so"
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", str(out),
                    os.path.join(ROOT, "tests", "nvtx_count.c"), "-lpthread"], check=True)
    return str(out)


def run_child(injection, body):
    """Run `body` (Python) in a child with the injection library; it has `pdv`
    and `counts()` in scope and prints one JSON line."""
    script = "\n".join([
        "import ctypes as C, json, sys",
        "sys.path.insert(0, %r)" % ROOT,
        "from paper_2012_00963_gb300 import pdv",
        "def counts(*names):",
        "    L = C.CDLL(%r)" % injection,
        "    L.nvtx_count_of.argtypes = [C.c_char_p]",
        "    d = {n: L.nvtx_count_of(n.encode()) for n in names}",
        "    d['_pushes'], d['_pops'], d['_unbalanced'] = L.nvtx_pushes(), L.nvtx_pops(), L.nvtx_unbalanced()",
        "    return d",
        body,
    ])
    env = dict(os.environ, NVTX_INJECTION64_PATH=injection)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_api_calls_push_balanced_ranges(injection):
    """Host-only: the context call (which fails without a GPU, and succeeds
    with one) and an invalid spectrum call each push and pop their range."""
    got = run_child(injection, "\n".join([
        "try:",
        "    h = pdv.pdv_ctx_create(0)",
        "    pdv.pdv_ctx_destroy(h)",
        "except pdv.PdvError:",
        "    pass",
        "try:",
        "    pdv.lib().pdv_simulate_spectrum(None, None)",
        "except Exception:",
        "    pass",
        "print(json.dumps(counts('pdv_ctx_create', 'pdv_simulate_spectrum')))",
    ]))
    assert got["pdv_ctx_create"] == 1 and got["pdv_simulate_spectrum"] == 1, got
    assert got["_pushes"] == got["_pops"] and got["_unbalanced"] == 0, got


@pytest.mark.gpu
def test_spectrum_and_serving_ranges(injection):
    got = run_child(injection, "\n".join([
        "from paper_2012_00963_gb300 import workloads as W",
        "wl = W.cfg1(n_packets=20000)",
        "with pdv.Context(0) as ctx:",
        "    cloud = pdv.Cloud(ctx, wl)",
        "    pdv.simulate_spectrum(ctx, cloud, wl)",
        "    req = pdv.Request(cloud, wl)",
        "    t = pdv.pdv_submit(ctx.handle, req.c)",
        "    while pdv.pdv_poll(ctx.handle, t, 100000) != pdv.PDV_OK:",
        "        pass",
        "    cloud.close()",
        "print(json.dumps(counts('pdv_ctx_create', 'pdv_create_cloud', 'pdv_set_phase_table',",
        "    'pdv_simulate_spectrum', 'pdv transport launch', 'pdv normalise', 'pdv_submit',",
        "    'pdv_poll', 'pdv serving launch', 'pdv serving normalise', 'pdv_ctx_destroy')))",
    ]))
    for name in ("pdv_ctx_create", "pdv_create_cloud", "pdv_set_phase_table",
                 "pdv_simulate_spectrum", "pdv transport launch", "pdv normalise", "pdv_submit",
                 "pdv serving normalise", "pdv_ctx_destroy"):
        assert got[name] == 1, (name, got)
    assert got["pdv_poll"] >= 1 and got["pdv serving launch"] >= 1, got
    assert got["_pushes"] == got["_pops"] and got["_unbalanced"] == 0, got
