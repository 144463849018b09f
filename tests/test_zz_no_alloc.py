"""The allocation-free velocity sweep, vlasov_sweep_velocity_static.

Some callers cannot allocate device memory once they are running: a host framework
that owns every allocation, a process that reserves its whole memory budget at
start-up, an allocator that is closed after initialisation.  For them the library
offers one velocity sweep that creates no context and keeps its scratch in a static
device array of fixed size.  These tests call it through the C ABI and check it
against the context-based vlasov_sweep on the same input, twice in a row.  The file
is collected last so that a run that stops at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _same(a, b):
    # the same kernels with the same constants: equal bit for bit
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def _grid(B, shape, V):
    g = B.Grid()
    g.nx, g.ny, g.nz, g.nux, g.nuy, g.nuz = shape
    g.L, g.V, g.dtype = 1.0, V, B.F32
    return g


@pytest.mark.parametrize("axis", [3, 4, 5])
def test_static_sweep_matches_context_sweep_twice(axis):
    from paper_2110_15867_gb300 import binding as B
    B.load()
    n, nu, V = (6, 5, 7), (8, 20, 12), 5.0
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=7), I.fermi_dirac(nu, V), np.float32)
    phi = torch.from_numpy(I.fourier_potential(n, seed=8).astype(np.float32)).cuda()
    dts = [0.004, -0.003]
    ref = torch.from_numpy(f0).cuda()
    ctx = B.Vlasov(ref, V=V)
    out = torch.from_numpy(f0).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = _grid(B, out.shape, V)
    stream = torch.cuda.current_stream().cuda_stream
    for dt in dts:
        ctx.sweep(axis, dt, 1.0, phi)
        B.vlasov_sweep_velocity_static(g, out.data_ptr(), axis, dt, phi.data_ptr(),
                                       status.data_ptr(), stream)
        torch.cuda.synchronize()
        ctx.status()
        assert int(status.item()) == 0
        _same(out.cpu().numpy(), ref.cpu().numpy())
    ctx.close()


def test_static_sweep_without_status_word_and_limits():
    from paper_2110_15867_gb300 import binding as B
    B.load()
    shape, V = (4, 4, 4, 8, 8, 8), 5.0
    f0 = I.initial_f(I.gaussian_field(shape[:3], 0.05, seed=3), I.fermi_dirac(shape[3:], V),
                     np.float32)
    phi = torch.from_numpy(I.fourier_potential(shape[:3], seed=4).astype(np.float32)).cuda()
    ref = torch.from_numpy(f0).cuda()
    out = torch.from_numpy(f0).cuda()
    ctx = B.Vlasov(ref, V=V)
    g = _grid(B, shape, V)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        ctx.sweep(5, 0.01, 1.0, phi)
        B.vlasov_sweep_velocity_static(g, out.data_ptr(), 5, 0.01, phi.data_ptr(), None, stream)
    torch.cuda.synchronize()
    _same(out.cpu().numpy(), ref.cpu().numpy())
    ctx.close()
    # more spatial cells than the static scratch holds: rejected before any GPU work
    big = _grid(B, (64, 32, 32, 8, 8, 8), V)
    assert 64 * 32 * 32 > B.STATIC_MAX_CELLS
    with pytest.raises(B.VlasovError) as e:
        B.vlasov_sweep_velocity_static(big, out.data_ptr(), 3, 0.01, phi.data_ptr(), None, stream)
    assert e.value.code == B.EINVAL
    with pytest.raises(B.VlasovError) as e:
        B.vlasov_sweep_velocity_static(g, out.data_ptr(), 0, 0.01, phi.data_ptr(), None, stream)
    assert e.value.code == B.EINVAL
    # within the cell limit but too large for 32-bit tensor-map extents: rejected too
    wide = _grid(B, (4, 128, 64, 128, 128, 64), V)
    with pytest.raises(B.VlasovError) as e:
        B.vlasov_sweep_velocity_static(wide, out.data_ptr(), 4, 0.01, phi.data_ptr(), None, stream)
    assert e.value.code == B.EINVAL


def test_static_sweep_allocates_no_device_memory():
    # the point of the entry point: after a first call on each axis (which may load that
    # sweep's kernels on this device) further sweeps on every velocity axis leave the
    # device's free memory unchanged
    from paper_2110_15867_gb300 import binding as B
    B.load()
    shape, V = (8, 8, 8, 16, 16, 32), 5.0
    f0 = I.initial_f(I.gaussian_field(shape[:3], 0.05, seed=9), I.fermi_dirac(shape[3:], V),
                     np.float32)
    phi = torch.from_numpy(I.fourier_potential(shape[:3], seed=10).astype(np.float32)).cuda()
    out = torch.from_numpy(f0).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = _grid(B, shape, V)
    stream = torch.cuda.current_stream().cuda_stream
    for axis in (3, 4, 5):
        B.vlasov_sweep_velocity_static(g, out.data_ptr(), axis, 0.002, phi.data_ptr(), status.data_ptr(), stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for axis in (3, 4, 5):
            B.vlasov_sweep_velocity_static(g, out.data_ptr(), axis, 0.002, phi.data_ptr(), status.data_ptr(),
                                           stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(status.item()) == 0
