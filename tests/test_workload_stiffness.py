"""The batched workload's stiffness spread, measured on the oracle: the
bimodal temperature draw (700-900 K and 1800-2400 K) must spread the RKC
stage counts over 2..~200 and the per-cell cost over two orders of
magnitude, which is what a persistent launch with work redistribution has
to balance. Cold cells stay at the minimum stage count."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
from paper_1309_2710_gb300 import synth

NAME = "c2h4_111sp_rkc_batched"


def _trace(m, T, p, Y, dt):
    om = oracle.Mech(m)

    def one(c):
        _, st, tr = oracle.trace_cell(om, T[c], p[c], Y[:, c], dt, 1e-6, 1e-10, oracle.RKC_POWER,
                                      cap=200000)
        return st, tr["s"], int(tr["stats"][0])

    with ThreadPoolExecutor(8) as ex:  # the oracle's C code runs without the GIL
        return list(ex.map(one, range(T.shape[0])))


def test_stage_counts_span_two_to_about_two_hundred():
    m = synth.workload_mechanism(NAME)
    T, p, Y = synth.workload_states(NAME, m, cells=48, seed_offset=100)
    hot = T > 1300.0
    out = {}
    for dt in synth.WORKLOADS[NAME]["dt"]:
        res = _trace(m, T, p, Y, dt)
        assert all(r[0] == 0 for r in res)
        smax = np.array([r[1].max() for r in res])
        nfe = np.array([r[2] for r in res])
        out[dt] = (np.concatenate([r[1] for r in res]), smax, nfe)
        assert smax[~hot].max() <= 8  # cold cells: frozen chemistry, few stages
        assert smax[hot].min() >= 20
    s_all = np.concatenate([v[0] for v in out.values()])
    nfe = np.concatenate([v[2] for v in out.values()])
    print("stages %d..%d, f evaluations per cell %d..%d" % (s_all.min(), s_all.max(), nfe.min(), nfe.max()))
    assert s_all.min() == 2
    assert 150 <= s_all.max() <= 250
    assert nfe.max() >= 100 * nfe.min()
