"""The allocation-free entry point, rom_spectral_radius_noalloc.

It serves callers that cannot call cudaMalloc (a host that gives the library a
fixed memory budget, or code that must not grow the device footprint): its
work vectors sit in a fixed device array inside the library.  This file is
collected last so that a failure here, under `-x`, comes after every other
test has run.  It must pass on its own in a fresh process and after the rest.
"""
import numpy as np
import pytest

from paper_2009_11742_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_11742_gb300 import build
    build.build()
    from paper_2009_11742_gb300 import rom as R
    return R


def colmajor_device(A):
    """A column-major FP64 device copy of the logical matrix A."""
    return torch.as_tensor(np.ascontiguousarray(np.asarray(A, np.float64).T), device="cuda")


@pytest.mark.parametrize("Kv,Ks", [(300, 300), (96, 130)])
def test_noalloc_matches_rom_create_twice(rom, Kv, Ks):
    """Two calls in a row agree with the spectral radius rom_create computes
    (same tolerance as the other spectral-radius checks); the second call
    reuses the shared work area the first one left behind."""
    p = inputs.make_problem(Kv, Ks, 1, 0, seed=Kv + Ks)
    h = rom.Rom.from_problem(p)
    ref = h.spectral_radius()
    Avs = colmajor_device(p.Avs)
    Asv = colmajor_device(p.Asv)
    for _ in range(2):
        st, rho = rom.rom_spectral_radius_noalloc(Avs.data_ptr(), Asv.data_ptr(), Kv, Ks, None)
        assert st == rom.ROM_OK
        assert abs(rho - ref) / ref < 1e-8
    h.close()


def test_noalloc_allocates_nothing(rom):
    """The point of the entry point: once the first call on the device has
    looked up the fixed work array, a call leaves the device's free memory
    and torch's allocator exactly as they were."""
    Kv, Ks = 256, 200
    p = inputs.make_problem(Kv, Ks, 1, 0, seed=11)
    Avs = colmajor_device(p.Avs)
    Asv = colmajor_device(p.Asv)
    st, rho0 = rom.rom_spectral_radius_noalloc(Avs.data_ptr(), Asv.data_ptr(), Kv, Ks, None)
    assert st == rom.ROM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    st, rho1 = rom.rom_spectral_radius_noalloc(Avs.data_ptr(), Asv.data_ptr(), Kv, Ks, None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == rom.ROM_OK and rho1 == rho0
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_reports_no_convergence(rom):
    """A product Avs Asv whose dominant eigenvalues are the complex pair +-2i
    of a non-normal 2 x 2 matrix: the power iteration's estimates alternate
    between two values and never settle, so the call says so instead of
    returning the last estimate as a result."""
    # keep both device copies alive for the call: a temporary's memory goes
    # back to torch's cache at once and the second copy could reuse it
    Avs = colmajor_device(np.eye(2))
    Asv = colmajor_device(np.array([[0.0, -4.0], [1.0, 0.0]]))
    st, rho = rom.rom_spectral_radius_noalloc(Avs.data_ptr(), Asv.data_ptr(), 2, 2, None)
    assert st == rom.ROM_E_NOCONV
    assert np.isfinite(rho)


def test_noalloc_refuses_oversize_and_host_buffers(rom):
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    st, _ = rom.rom_spectral_radius_noalloc(x.data_ptr(), x.data_ptr(), 4097, 4, None)
    assert st == rom.ROM_E_INVAL
    hostbuf = np.zeros(16)
    st, _ = rom.rom_spectral_radius_noalloc(hostbuf.ctypes.data, hostbuf.ctypes.data, 4, 4, None)
    assert st == rom.ROM_E_INVAL
