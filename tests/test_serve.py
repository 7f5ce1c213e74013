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
    srv = serve.Server(groups, budget_bytes=1 << 30, slots_per_group=2)
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
    """The budget holds the slots' workspaces plus the device state of the
    admitted requests. With room for the largest request only, two requests
    are resident at the same time only if both fit together, and the
    resident bytes never exceed what the workspaces leave of the budget."""
    groups, pools = setup
    reqs = _requests(pools, 12, seed=2)
    probe = serve.Server(groups, 1 << 40, slots_per_group=2)
    probe._size_workspaces(reqs)
    ws = probe.ws_bytes
    assert ws > 0
    room = max(probe.request_bytes(r) for r in reqs)
    srv = serve.Server(groups, budget_bytes=ws + room, slots_per_group=2)
    out = srv.run(reqs)
    for r in out:
        assert r.status.max().item() == 0
    assert srv.used == 0
    assert srv.ws_bytes == ws
    assert 0 < srv.peak_used <= room
    together = 0
    for a in out:
        for b in out:
            if a.rid < b.rid and a.t_admit < b.t_done and b.t_admit < a.t_done:
                together += 1
                assert srv.request_bytes(a) + srv.request_bytes(b) <= room
    # and the rule is not vacuous: some pair did not fit together
    pairs = [(a, b) for a in out for b in out if a.rid < b.rid]
    assert any(srv.request_bytes(a) + srv.request_bytes(b) > room for a, b in pairs)
    with pytest.raises(ValueError):
        serve.Server(groups, budget_bytes=ws + room - 1, slots_per_group=2).run(reqs)


def test_one_launch_per_request_matches(setup):
    groups, pools = setup
    reqs = _requests(pools, 6, seed=3)
    out = serve.one_launch_per_request(groups, reqs)
    for r in out:
        Ya, _ = _alone(groups, r)
        assert torch.equal(r.Y_out, Ya)
