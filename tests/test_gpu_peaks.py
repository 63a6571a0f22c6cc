"""The throughput probes behind the roofline peaks that the copy and GEMM
benchmarks do not give: the probe program runs to completion, every bounded
wait completes, and its tcgen05 MMAs (kind::f8f6f4, kind::mxf4 and
kind::mxf4nvf4 with unit scale factors) reproduce a 0/1 integer product bit
for bit before they are timed."""
import json
import os
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0811_1714_gb300 import buildlib  # noqa: E402


def test_peak_probes_run_and_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    buildlib.build()
    exe = buildlib.probe_path("peaks")
    assert os.path.exists(exe)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    p = json.loads(r.stdout.strip().splitlines()[-1])
    assert p["l2_tma_status"] == 0
    for key in ("tcgen05_f8f6f4_m128n256", "tcgen05_mxf4_m128n256", "tcgen05_mxf4_m128n128",
                "tcgen05_f8f6f4_m128n128", "tcgen05_mxf4nvf4_4x_m128n256"):
        assert p[key]["wrong"] == 0 and p[key]["status"] == 0, (key, p[key])
        assert p[key]["tflops"] > 0
    assert p["tcgen05_mxf4_a_in_tmem_m128n256"]["status"] == 0
    assert p["smem_lookup_tbs"] > 0 and p["mma_sync_s8_tops"] > 0
