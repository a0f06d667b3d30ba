"""The C ABI from C: tests/gpu_src/abi_client.c includes only include/rlb.h, links librlb.so and runs two tubes
(the paper's Sod tube and a ballistic one) in one handle. Its fields after the run must equal, bit for bit,
those of the same run through the Python binding; it also checks a restart from a checkpoint and that bad
arguments come back as RLB_EINVAL."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1608_03004_gb300 import binding as rb
from paper_1608_03004_gb300 import build as B

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_c_client_matches_the_python_binding():
    lib = rb.library_path()
    rb.load()  # builds the library if needed
    work = tempfile.mkdtemp(prefix="rlb_c_")
    try:
        exe = os.path.join(work, "abi_client")
        subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(B.ROOT, "include"),
                        os.path.join(HERE, "gpu_src", "abi_client.c"), "-o", exe, lib,
                        "-Wl,-rpath," + os.path.dirname(lib), "-lm"], check=True)
        out = os.path.join(work, "fields.bin")
        nsteps = 40
        r = subprocess.run([exe, str(nsteps), out], capture_output=True, text=True, timeout=300)
        print(r.stdout, r.stderr)
        assert r.returncode == 0, r.stderr
        assert "restart repeats the run: yes" in r.stdout
        assert "negative nsteps: EINVAL" in r.stdout and "bad orders: EINVAL" in r.stdout
        got = np.fromfile(out, dtype=np.float64).reshape(rb.NFIELDS, 400 + 257)
    finally:
        shutil.rmtree(work, ignore_errors=True)
    t0 = rb.Tube.make(400, 8, 1e-3)
    t1 = rb.Tube.make(257, 32, float("inf"))
    states = np.array([[1.0, 1.0, 0.0, 0.1, 0.125, 0.0]] * 2)
    with rb.rlb_init_riemann([t0, t1], states, np.array([-0.5, -0.5])) as h:
        rb.rlb_step(h, nsteps)
        ref = rb.rlb_moments(h)
    np.testing.assert_array_equal(got, ref)
