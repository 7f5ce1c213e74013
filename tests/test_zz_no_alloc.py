"""kin_integrate_noalloc, the entry point for callers that cannot allocate
device memory when they integrate (their working memory comes from a fixed
array the library reserves per device). Checked through the C ABI against
kin_integrate, which uses a caller workspace, on two calls in a row. This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import kin, synth  # noqa: E402
from tests.parity import compare  # noqa: E402

DEV = torch.device("cuda:0")
NAME = "h2co_13sp_rkc"


def _run(fn_name, km, T, p, Y, dt, ws=None):
    cells = T.shape[0]
    Td = torch.as_tensor(T, device=DEV)
    pd = torch.as_tensor(p, device=DEV)
    Yd = torch.as_tensor(np.ascontiguousarray(Y), device=DEV)
    st = torch.zeros(cells, dtype=torch.uint8, device=DEV)
    sta = torch.zeros((cells, kin.NSTATS), dtype=torch.int32, device=DEV)
    o = kin.Opts(kin.RKC, kin.FP64, 0, 0, 0, 0, 0, 0, kin.LAYOUT_AUTO, 0, kin.FEVAL_AUTO,
                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    args = [km.handle, cells, kin._ptr(Td), kin._ptr(pd), kin._ptr(Yd), cells, dt, 1e-6, 1e-10,
            ctypes.byref(o), kin._ptr(st), kin._ptr(sta)]
    if fn_name == "kin_integrate":
        args += [kin._ptr(ws), ws.numel()]
    rc = getattr(kin.lib(), fn_name)(*args)
    assert rc == kin.KIN_OK, kin.lib().kin_last_error()
    torch.cuda.synchronize()
    return Yd.cpu().numpy(), st.cpu().numpy(), sta.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice():
    m = synth.workload_mechanism(NAME)
    km = kin.Mechanism(m)
    for cells, dt, seed in ((20000, 1e-6, 41), (3001, 3e-7, 42)):
        T, p, Y = synth.workload_states(NAME, m, cells=cells, seed_offset=seed)
        ws = km.workspace(kin.RKC, kin.FP64, cells)
        Ya, sa, xa = _run("kin_integrate", km, T, p, Y, dt, ws)
        Yb, sb, xb = _run("kin_integrate_noalloc", km, T, p, Y, dt)
        assert (sa == 0).all()
        compare(Yb, Ya, sb, sa, xb, xa, 1e-10, 1e-6)


def test_noalloc_rejects_cells_beyond_the_fixed_array():
    m = synth.workload_mechanism(NAME)
    km = kin.Mechanism(m)
    one = torch.zeros(1, dtype=torch.float64, device=DEV)
    Y = torch.zeros((m.n_species, 1), dtype=torch.float64, device=DEV)
    o = kin.Opts(kin.RKC, kin.FP64, 0, 0, 0, 0, 0, 0, kin.LAYOUT_AUTO, 0, kin.FEVAL_AUTO, None)
    # 10 million cells cannot fit in 64 MiB: refused before any launch or
    # pointer use
    rc = kin.lib().kin_integrate_noalloc(km.handle, 10_000_000, kin._ptr(one), kin._ptr(one),
                                         kin._ptr(Y), 10_000_000, 1e-6, 1e-6, 1e-10,
                                         ctypes.byref(o), None, None)
    assert rc == kin.KIN_ENOMEM
    assert b"fixed array" in kin.lib().kin_last_error()
