"""The reversible -> irreversible conversion (Appendix A) end to end on the
GPU: a converted mechanism (13 species, 27 reversible reactions -> 54
irreversible, the paper's H2/CO counts) integrated through the C ABI against
the oracle on the same converted tables, and a converted pair reaching its
thermodynamic equilibrium."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1309_2710_gb300 import irrev, synth  # noqa: E402
from tests import mechs  # noqa: E402
from tests.parity import compare  # noqa: E402

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import kin  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def converted_h2co():
    m = synth.make_reversible_mechanism(13, 27, ("H", "O", "C", "N"), tb_frac=0.1, seed=1102)
    return irrev.to_irreversible(m, np.ones(27, bool))


@pytest.mark.parametrize("energy,layout", [(0, kin.LAYOUT_LANE), (1, kin.LAYOUT_LANE),
                                           (0, kin.LAYOUT_WARP)])
def test_converted_mechanism_against_oracle(energy, layout):
    mi = converted_h2co()
    assert len(mi.lnA) == 54
    km, om = kin.Mechanism(mi), oracle.Mech(mi)
    # hot cells and a long flow step, so that the reverse reactions matter
    T, p, Y = synth.make_states(mi, 300, T_range=(1800.0, 2800.0), seed=2102)
    Td, Yd = dev(T), dev(Y)
    st = torch.zeros(300, dtype=torch.uint8, device=DEV)
    sta = torch.zeros((300, kin.NSTATS), dtype=torch.int32, device=DEV)
    kin.integrate(km, Td, dev(p), Yd, 1e-4, 1e-6, 1e-10, kin.RKC, status=st, stats=sta,
                  sigma=kin.SIGMA_POWER, energy=energy, layout=layout, max_steps=20000)
    torch.cuda.synchronize()
    r = oracle.integrate(om, T, p, Y, 1e-4, 1e-6, 1e-10, oracle.RKC_POWER, energy=bool(energy),
                         max_steps=20000)
    assert (r[1] == 0).all()
    Yg, Yo = Yd.cpu().numpy(), r[0]
    if energy:
        Yg, Yo = np.vstack([Yg, Td.cpu().numpy()]), np.vstack([Yo, r[4]])
    s = compare(Yg, Yo, st.cpu().numpy(), r[1], sta.cpu().numpy(), r[2], 1e-10, 1e-6,
                max_div_frac=0.05)
    print("converted h2co", energy, layout, s)


def test_converted_pair_reaches_equilibrium_on_the_gpu():
    cp, Hf, S0 = [30.0, 36.0], [0.0, -8e3], [200.0, 190.0]
    m = mechs.mech([28.0, 28.0], [dict(reac=[0], prod=[1], A=2e6, beta=0.3, Ea=2e4)],
                   cp=cp, Hf=Hf, S0=S0)
    km = kin.Mechanism(irrev.to_irreversible(m, [True]))
    T = 1000.0
    Kc = irrev.equilibrium_constant(cp, Hf, S0, [0], [1], T)
    kf = 2e6 * T ** 0.3 * math.exp(-2e4 / (8.314462618 * T))
    cells = 64
    Y = np.zeros((2, cells))
    Y[0] = np.linspace(0.05, 0.95, cells)
    Y[1] = 1.0 - Y[0]
    Yd = dev(Y)
    kin.integrate(km, dev(np.full(cells, T)), dev(np.full(cells, 101325.0)), Yd,
                  40.0 / (kf * (1 + 1 / Kc)), 1e-10, 1e-14, kin.RKCK)
    torch.cuda.synchronize()
    Yn = Yd.cpu().numpy()
    np.testing.assert_allclose(Yn[1] / Yn[0], Kc, rtol=1e-7)
