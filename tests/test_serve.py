"""Serving: continuous batching returns, for every request, exactly what the
request gets when it is integrated alone, while requests overlap on the
device; admission respects the memory budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import kin, serve, synth  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    groups, pools = {}, {}
    for name in ("h2co_13sp_rkc", "ch4_53sp_rkc_mixed"):
        w = synth.WORKLOADS[name]
        m = synth.workload_mechanism(name)
        groups[name] = serve.Group(kin.Mechanism(m), w["method"], w["precision"],
                                   dict(serve.SERVE_SHAPES[name]), w["sigma"])
        pools[name] = serve.StatePool(name, m, 8192, seed_offset=900)
    return groups, pools


def _requests(pools, n, seed, rate=None):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(n):
        g = "h2co_13sp_rkc" if rng.uniform() < 0.5 else "ch4_53sp_rkc_mixed"
        cells = int(np.exp(rng.uniform(np.log(64), np.log(3000))))
        dt = float(np.exp(rng.uniform(np.log(1e-7), np.log(3e-6))))
        off = int(rng.integers(0, pools[g].cells - cells + 1))
        T, p, Y = pools[g].view(off, cells)
        if rate:
            t += rng.exponential(1.0 / rate)
        out.append(serve.Request(i, g, T, p, Y, dt, arrival=t))
    return out


def _alone(groups, r):
    g = groups[r.group]
    d = torch.device("cuda")
    Yd = r.Y.to(d).contiguous()
    st = torch.empty(r.cells, dtype=torch.uint8, device=d)
    kin.integrate(g.mech, r.T.to(d), r.p.to(d), Yd, r.dt, r.rtol, r.atol, g.method, g.precision,
                  status=st, sigma=g.sigma, layout=g.shape.get("layout", kin.LAYOUT_AUTO),
                  feval=g.shape.get("feval", kin.FEVAL_AUTO))
    torch.cuda.synchronize()
    return Yd.cpu(), st.cpu()


def test_served_equals_alone(setup):
    groups, pools = setup
    reqs = _requests(pools, 40, seed=1, rate=400.0)
    srv = serve.Server(groups, budget_bytes=64 << 20, slots_per_group=2)
    out = srv.run(reqs)
    assert srv.used == 0
    launched_while_busy = 0
    for r in out:
        Ya, sa = _alone(groups, r)
        assert torch.equal(r.Y_out, Ya), r.rid
        assert torch.equal(r.status, sa)
        assert r.t_done >= r.t_launch >= r.t_admit >= r.arrival
    # some request was launched while another one was still running
    iv = sorted((r.t_launch, r.t_done) for r in out)
    for i in range(1, len(iv)):
        if iv[i][0] < max(e for _, e in iv[:i]):
            launched_while_busy += 1
    assert launched_while_busy > 0


def test_budget_limits_resident_state(setup):
    groups, pools = setup
    reqs = _requests(pools, 12, seed=2)
    budget = max(serve.Server(groups, 1).request_bytes(r) for r in reqs)
    srv = serve.Server(groups, budget_bytes=budget, slots_per_group=2)
    out = srv.run(reqs)
    # with room for only the largest request, admissions serialise: a request
    # is admitted only after the previous admitted one completed, unless both fit
    for r in out:
        assert r.status.max().item() == 0
    assert srv.used == 0


def test_one_launch_per_request_matches(setup):
    groups, pools = setup
    reqs = _requests(pools, 6, seed=3)
    out = serve.one_launch_per_request(groups, reqs)
    for r in out:
        Ya, _ = _alone(groups, r)
        assert torch.equal(r.Y_out, Ya)
