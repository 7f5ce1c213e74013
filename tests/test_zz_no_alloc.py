"""kin_integrate_noalloc, the entry point for callers that cannot allocate
device memory when they integrate (a flow solver whose memory manager owns
every device byte, or code running where allocation is forbidden): its
working memory comes from a fixed array the library reserves per device.

Checked through the C ABI against kin_integrate, which takes a caller
workspace, on two calls in a row. Both run the same kernels on the same
inputs, so results, status and statistics must match bit for bit; a call
that reused stale contents of the shared array would show here. Free device
memory is read around a call to show that the call allocates nothing. This
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

DEV = torch.device("cuda:0")
NAME = "h2co_13sp_rkc"


def _opts(feval=kin.FEVAL_AUTO, layout=kin.LAYOUT_AUTO, blocks_per_sm=0, block_threads=0):
    return kin.Opts(kin.RKC, kin.FP64, 0, block_threads, blocks_per_sm, 0, 0, 0, layout, 0, feval,
                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _run(fn_name, km, T, p, Y, dt, o, ws=None, free_check=False):
    """One call through the C ABI; returns (Y, status, stats) and, with
    free_check, the change of free device memory across the call."""
    cells = T.shape[0]
    Td = torch.as_tensor(T, device=DEV)
    pd = torch.as_tensor(p, device=DEV)
    Yd = torch.as_tensor(np.ascontiguousarray(Y), device=DEV)
    st = torch.full((cells,), 255, dtype=torch.uint8, device=DEV)
    sta = torch.full((cells, kin.NSTATS), -1, dtype=torch.int32, device=DEV)
    args = [km.handle, cells, kin._ptr(Td), kin._ptr(pd), kin._ptr(Yd), cells, dt, 1e-6, 1e-10,
            ctypes.byref(o), kin._ptr(st), kin._ptr(sta)]
    if fn_name == "kin_integrate":
        args += [kin._ptr(ws), ws.numel()]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc = getattr(kin.lib(), fn_name)(*args)
    assert rc == kin.KIN_OK, kin.lib().kin_last_error()
    torch.cuda.synchronize()
    dfree = torch.cuda.mem_get_info()[0] - free0
    out = (Yd.cpu().numpy(), st.cpu().numpy(), sta.cpu().numpy())
    return out + ((dfree,) if free_check else ())


def _assert_same(a, b):
    assert np.array_equal(a[0], b[0]), np.abs(a[0] - b[0]).max()
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


def test_noalloc_matches_workspace_entry_point_twice():
    m = synth.workload_mechanism(NAME)
    km = kin.Mechanism(m)
    for k, (cells, dt, seed) in enumerate(((20000, 1e-6, 41), (3001, 3e-7, 42))):
        T, p, Y = synth.workload_states(NAME, m, cells=cells, seed_offset=seed)
        ws = km.workspace(kin.RKC, kin.FP64, cells)
        a = _run("kin_integrate", km, T, p, Y, dt, _opts(), ws)
        b = _run("kin_integrate_noalloc", km, T, p, Y, dt, _opts(), free_check=k == 1)
        assert (a[1] == 0).all() and (b[1] == 0).all()
        _assert_same(a, b)
        if k == 1:
            # the second call: kernels and the fixed array are loaded already
            assert b[3] == 0, "free device memory changed by %d bytes" % b[3]


def test_noalloc_all_lanes_when_blocks_per_sm_is_zero():
    """blocks_per_sm = 0 resolves as in kin_integrate (as many as fit: 16
    blocks of 32 lanes per SM), stepping down only as far as the fixed array
    needs. Launch shapes give the same bits, so the result equals the
    workspace call's."""
    m = synth.workload_mechanism(NAME)
    km = kin.Mechanism(m)
    T, p, Y = synth.workload_states(NAME, m, cells=12000, seed_offset=43)
    o = _opts(layout=kin.LAYOUT_LANE, block_threads=32)
    ws = torch.empty(kin.lib().kin_workspace_bytes(km.handle, ctypes.byref(o), 12000),
                     dtype=torch.uint8, device=DEV)
    a = _run("kin_integrate", km, T, p, Y, 1e-6, o, ws)
    b = _run("kin_integrate_noalloc", km, T, p, Y, 1e-6, _opts(layout=kin.LAYOUT_LANE, block_threads=32))
    _assert_same(a, b)


def test_noalloc_never_compiles_the_generated_f():
    """A mechanism whose generated f no call has loaded: the automatic choice
    takes the tables (the same bits as kin_integrate with the tables), a
    forced generated f is refused before any launch. Once kin_integrate has
    compiled and loaded it, the no-allocation call runs it, with the same
    bits as kin_integrate, and free memory stays put."""
    m = synth.make_mechanism(6, 20, ("H", "O"), tb_frac=0.1, seed=9177)  # used by no other test
    km = kin.Mechanism(m)
    cells = 70000  # above KIN_GEN_MIN_CELLS: kin_integrate's automatic choice is the generated f
    T, p, Y = synth.make_states(m, cells, T_range=(1200.0, 1800.0), seed=9178)
    lane = dict(layout=kin.LAYOUT_LANE)
    o_tab = _opts(feval=kin.FEVAL_TABLE, **lane)
    ws = torch.empty(kin.lib().kin_workspace_bytes(km.handle, ctypes.byref(o_tab), cells),
                     dtype=torch.uint8, device=DEV)
    a = _run("kin_integrate", km, T, p, Y, 1e-6, o_tab, ws)
    b = _run("kin_integrate_noalloc", km, T, p, Y, 1e-6, _opts(feval=kin.FEVAL_AUTO, **lane))
    _assert_same(a, b)
    dummy = torch.zeros(1, dtype=torch.float64, device=DEV)
    Yd = torch.zeros((m.n_species, 1), dtype=torch.float64, device=DEV)
    rc = kin.lib().kin_integrate_noalloc(km.handle, 1, kin._ptr(dummy), kin._ptr(dummy), kin._ptr(Yd), 1,
                                         1e-6, 1e-6, 1e-10,
                                         ctypes.byref(_opts(feval=kin.FEVAL_GENERATED, **lane)), None, None)
    assert rc == kin.KIN_EUNSUPPORTED
    assert b"not loaded" in kin.lib().kin_last_error()
    o_gen = _opts(feval=kin.FEVAL_GENERATED, **lane)
    a = _run("kin_integrate", km, T, p, Y, 1e-6, o_gen, ws)  # compiles and loads
    b = _run("kin_integrate_noalloc", km, T, p, Y, 1e-6, o_gen, free_check=True)
    _assert_same(a, b[:3])
    assert b[3] == 0, "free device memory changed by %d bytes" % b[3]


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
