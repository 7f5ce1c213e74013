"""The divergence study on the GPU (Section 3.1): per-cell f-evaluation counts
summed over consecutive flow steps, as the kernels report them, against the
oracle's counts for the same cells and steps; the warp measure D computed
from both; and the benchmark's divergence mode end to end."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1309_2710_gb300 import divergence as dv  # noqa: E402
from paper_1309_2710_gb300 import synth  # noqa: E402

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import kin  # noqa: E402

DEV = torch.device("cuda:0")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def omethod(w):
    if w["method"] == kin.RKCK:
        return oracle.RKCK
    return oracle.RKC_POWER if w["sigma"] == kin.SIGMA_POWER else oracle.RKC


@pytest.mark.parametrize("name,layout", [("h2_9sp_rkck", kin.LAYOUT_LANE),
                                         ("h2_9sp_rkck", kin.LAYOUT_WARP),
                                         ("h2co_13sp_rkc", kin.LAYOUT_LANE)])
def test_summed_counts_and_D_match_the_oracle(name, layout):
    w = synth.WORKLOADS[name]
    m = synth.workload_mechanism(name)
    km, om = kin.Mechanism(m), oracle.Mech(m)
    cells, steps = 1000, 3
    T, p, Y = synth.workload_states(name, m, cells=cells, seed_offset=71)
    Td, pd, Yd = (torch.as_tensor(np.ascontiguousarray(a), device=DEV) for a in (T, p, Y))
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=DEV)
    st = torch.zeros(cells, dtype=torch.uint8, device=DEV)
    d_gpu = np.zeros(cells, dtype=np.int64)
    d_orc = np.zeros(cells, dtype=np.int64)
    Yo = Y.copy()
    for _ in range(steps):
        kin.integrate(km, Td, pd, Yd, w["dt"], w["rtol"], w["atol"], w["method"], status=st, stats=sta,
                      sigma=w["sigma"], layout=layout)
        torch.cuda.synchronize()
        assert int(st.max()) == 0
        d_gpu += sta[:, 0].cpu().numpy()
        Yo, sto, stao, _ = oracle.integrate(om, T, p, Yo, w["dt"], w["rtol"], w["atol"], omethod(w))
        assert (sto == 0).all()
        d_orc += stao[:, 0]
    # the counts are the discrete trace of each cell: equal wherever the GPU
    # took the oracle's decisions (all but a few cells)
    same = d_gpu == d_orc
    assert same.mean() >= 0.97, same.mean()
    Dg = dv.warp_D(d_gpu)
    Do = dv.warp_D(d_orc)
    assert np.abs(Dg - Do).max() < 0.05
    assert abs(dv.lane_efficiency(d_gpu) - dv.lane_efficiency(d_orc)) < 0.01


def test_bench_divergence_mode_runs():
    cmd = [sys.executable, "bench.py", "--mode", "divergence", "--workload", "h2_9sp_rkck", "--cells", "2048",
           "--global-steps", "2", "--warmup", "1", "--no-tune"]
    out = subprocess.run(cmd, cwd=ROOT, check=True, capture_output=True, text=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["mode"] == "divergence" and line["cells"] == 2048 and line["global_steps"] == 2
    for order in ("similar", "random"):
        r = line[order]
        assert r["nonzero_status"] == 0 and len(r["ms_per_call"]) == 2
        D = r["D"]
        assert D["given_order"]["warps"] == 64 and sum(D["given_order"]["hist"]) == 64
        assert D["sorted_by_count"]["lane_efficiency"] >= D["given_order"]["lane_efficiency"]
