"""Device memory through the bem_create allocator hooks: with PyTorch's caching allocator as
the provider (the binding's default), every device byte a handle uses comes from the hook and
is handed back by bem_destroy, and the library allocates nothing on its own beside it."""
import numpy as np
import pytest
import torch

from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(bem, prec, N=2048, memory="torch"):
    v, _, _ = I.equal_chord_mesh(I.random_star(5), N)
    s = bem.Solver(device=0, prec=prec, memory=memory)
    s.assemble(torch.from_numpy(v).cuda(), 1.5, ops="SW")
    s.filter_apply(41)
    s.compress(1e-10)
    s.factor()
    vv = s.rhs_planewave(torch.from_numpy(I.planewave_angles(16)).cuda())
    x, it, res = s.solve(vv, report=True)
    torch.cuda.synchronize()
    return s, x, res


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_buffer_comes_from_the_hooks_and_goes_back(prec):
    from paper_2210_08580_gb300 import bem
    _run(bem, prec)[0].close()                      # loads every kernel of the path once
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    s, x, res = _run(bem, prec)
    mem = s.memory
    N = 2048
    assert mem.calls > 0
    assert mem.peak >= 2 * 16 * N * N               # S and N (complex128) at least
    free1, _ = torch.cuda.mem_get_info()
    grown_torch = torch.cuda.memory_reserved() - reserved0
    used_device = free0 - free1
    # whatever the device lost is accounted for by PyTorch's pool (a library cudaMalloc of
    # one N x N matrix would be 64 MiB)
    assert used_device <= grown_torch + (8 << 20), (used_device, grown_torch)
    held = mem.allocated
    assert held > 0
    s.close()
    assert mem.allocated == 0 and not mem.sizes, (mem.allocated, len(mem.sizes))
    assert res <= 1e-10


def test_hooked_and_runtime_memory_give_the_same_bits():
    from paper_2210_08580_gb300 import bem
    s1, x1, _ = _run(bem, "fp64", N=512, memory="torch")
    s2, x2, _ = _run(bem, "fp64", N=512, memory="cuda")
    assert torch.equal(x1, x2)
    assert s2.memory is None
    s1.close(); s2.close()


def test_one_hook_without_the_other_is_rejected():
    import ctypes
    from paper_2210_08580_gb300 import bem
    L = bem.load_library()
    mem = bem.TorchDeviceMemory(0, lambda: torch.cuda.current_stream())
    h = ctypes.c_void_p()
    st = L.bem_create(ctypes.byref(h), 0, None, None, mem.alloc_fn, bem.FREE_FN(), None)
    assert st == 1 and not h.value


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_refused_allocation_is_reported_and_recoverable(prec):
    """Allocation failure injected on the host (the provider refuses every request after the
    first n): for each n up to the path's last allocation, the failing call returns
    BEM_E_NOMEM, the same handle then runs the whole path once the provider serves again and
    gives the bits of a handle that never failed, and bem_destroy hands back every byte."""
    from paper_2210_08580_gb300 import bem
    v, _, _ = I.equal_chord_mesh(I.random_star(5), 1024)
    vd = torch.from_numpy(v).cuda()
    ang = torch.from_numpy(I.planewave_angles(16)).cuda()

    def path(s):
        s.assemble(vd, 1.5, ops="SW")
        s.filter_apply(41)
        s.compress(1e-10)
        s.factor()
        x = s.solve(s.rhs_planewave(ang))
        torch.cuda.synchronize()
        return x

    ref = bem.Solver(device=0, prec=prec)
    x_ref = path(ref)
    ref.close()
    failed = 0
    for n in range(400):
        s = bem.Solver(device=0, prec=prec)
        mem = s.memory
        mem.fail_after = n
        try:
            path(s)
            clean = True
        except bem.BemError as e:
            assert e.status == 2, (n, str(e))
            clean = False
        torch.cuda.synchronize()
        if not clean:
            failed += 1
            assert mem.refused >= 1
            mem.fail_after = None
            assert torch.equal(path(s), x_ref), n
        s.close()
        assert mem.allocated == 0 and not mem.sizes, (n, mem.allocated)
        if clean:
            break
    assert clean and failed >= 5, (failed, n)
