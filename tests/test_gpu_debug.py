"""The debug build (libpdv_debug.so, index checks in the kernels and path
traces): its cases (tests/debug_build_cases.py) run in a child process that
loads it through PDV_LIBRARY=debug. The release library, loaded here, has no
checks: it reports debug_build 0 and refuses the debug-only calls."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2012_00963_gb300 import pdv
from paper_2012_00963_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_cases():
    env = dict(os.environ, PDV_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x",
                        os.path.join(ROOT, "tests", "debug_build_cases.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=3000)
    print(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-6000:] + r.stderr[-3000:]


def test_release_library_has_no_checks():
    assert pdv.library_path().endswith("libpdv.so")
    with pdv.Context(0) as ctx:
        d = pdv.pdv_debug_get(ctx.handle, reset=True)
        assert d["debug_build"] == 0 and d["violations"] == 0
        with pytest.raises(pdv.PdvError) as e:
            pdv.pdv_debug_set_trace(ctx.handle, 4, 4, np.zeros((4, 4), pdv.TRACE_DTYPE))
        assert e.value.status == pdv.PDV_EINVAL
        wl = W.cfg1(n_packets=1000)
        cloud = pdv.Cloud(ctx, wl)
        with pytest.raises(pdv.PdvError) as e:
            pdv.simulate_spectrum(ctx, cloud, wl, debug_check=True)
        assert e.value.status == pdv.PDV_EINVAL
        cloud.close()
