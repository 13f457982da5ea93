"""RS / VRS forwards that keep the spectra of their zero-padded inputs, and the adjoints that use
them.

The saved-spectrum entry points compute what xl_rs_propagate / xl_vrs_propagate and their
adjoints compute: the forwards and the adjoints' field gradients with the same kernels on the same
values (compared bit for bit), the distance gradient from the saved spectra instead of transforming
the input again (the same products, summed in another kernel: compared to rounding). The plain
entry points are compared with the FP64 oracle in test_gpu_rs.py; one case per precision also
goes to the oracle directly here.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C64, TOL_C128, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu
LAM = 0.6328


def _grid(n, pitch):
    return inputs.Grid(n, n, pitch, pitch, -(n // 2) * pitch, -(n // 2) * pitch)


def _fields(n, comps, batch, seed, dtype):
    g = _grid(n, 1.0)
    us = []
    for b in range(batch):
        planes = [inputs.gaussian_random_phase(g, 0.3 * n, seed + 10 * b + c) for c in range(comps)]
        us.append(np.stack(planes) if comps > 1 else planes[0])
    return g, np.ascontiguousarray(np.stack(us).astype(dtype))


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_rs_saved_bit_identical(dtype):
    import torch
    xl = lib()
    g, u = _fields(128, 1, 3, 4100, dtype)
    zs = [500.0, 500.0, 2000.0]  # two launches: a run of equal distances, then one more
    U = to_dev(u, dtype)
    out_plain = xl.rs_propagate(U, g, LAM, zs)
    S = xl.save_buffer(U)
    out_save = xl.rs_propagate(U, g, LAM, zs, saved=S)
    assert torch.equal(out_plain, out_save)
    G = to_dev(inputs.random_unit(4101, (3, 128, 128)).astype(dtype), dtype)
    gi_p, gz_p = xl.rs_propagate_backward(G, U, g, LAM, zs, want_field=True, want_dz=True)
    gi_s, gz_s = xl.rs_propagate_backward(G, None, g, LAM, zs, want_field=True, want_dz=True,
                                          saved=S)
    assert torch.equal(gi_p, gi_s)
    assert torch.allclose(gz_p, gz_s, rtol=1e-5 if dtype == np.complex64 else 1e-12, atol=0)
    # only the distance gradient
    _, gz_o = xl.rs_propagate_backward(G, None, g, LAM, zs, want_field=False, want_dz=True, saved=S)
    assert np.allclose(to_np(gz_o), to_np(gz_s), rtol=1e-12 if dtype == np.complex128 else 1e-6)
    # the oracle, element 2
    u2 = u[2].astype(np.complex128)
    ref = oracle.rs_conv(u2, g.dx, g.dy, LAM, zs[2])
    assert rel(to_np(out_save)[2], ref) < (TOL_C64 if dtype == np.complex64 else TOL_C128)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_vrs_saved_bit_identical(dtype):
    import torch
    xl = lib()
    g, u = _fields(64, 2, 2, 4200, dtype)
    zs = [800.0, 300.0]
    U = to_dev(u, dtype)
    out_plain = xl.vrs_propagate(U, g, LAM, zs)
    S = xl.save_buffer(U, 2)
    out_save = xl.vrs_propagate(U, g, LAM, zs, saved=S)
    assert torch.equal(out_plain, out_save)
    G = to_dev(inputs.random_unit(4201, (2, 3, 64, 64)).astype(dtype), dtype)
    for pinv in (False, True):
        gi_p, gz_p = xl.vrs_propagate_backward(G, U, g, LAM, zs, want_field=True, want_dz=True,
                                               phase_invariant=pinv)
        gi_s, gz_s = xl.vrs_propagate_backward(G, None, g, LAM, zs, want_field=True, want_dz=True,
                                               phase_invariant=pinv, saved=S)
        assert torch.equal(gi_p, gi_s)
        assert torch.allclose(gz_p, gz_s, rtol=1e-5 if dtype == np.complex64 else 1e-12, atol=0)
    ref = oracle.vrs(u[1].astype(np.complex128), g.dx, g.dy, LAM, zs[1])
    assert rel(to_np(out_save)[1], ref) < (TOL_C64 if dtype == np.complex64 else TOL_C128)


def test_rs_saved_device_distances():
    """Device-resident (trainable) distances: one launch per element, same results."""
    import torch
    xl = lib()
    g, u = _fields(64, 1, 2, 4300, np.complex64)
    U = to_dev(u, np.complex64)
    zd = torch.tensor([700.0, 1500.0], dtype=torch.float64, device="cuda")
    S = xl.save_buffer(U)
    out_save = xl.rs_propagate(U, g, LAM, zd, saved=S)
    assert torch.equal(out_save, xl.rs_propagate(U, g, LAM, zd))
    G = to_dev(inputs.random_unit(4301, (2, 64, 64)).astype(np.complex64), np.complex64)
    gi_p, gz_p = xl.rs_propagate_backward(G, U, g, LAM, zd, want_field=True, want_dz=True)
    gi_s, gz_s = xl.rs_propagate_backward(G, None, g, LAM, zd, want_field=True, want_dz=True, saved=S)
    assert torch.equal(gi_p, gi_s)
    assert torch.allclose(gz_p, gz_s, rtol=1e-5, atol=0)


def test_saved_argument_errors():
    import torch
    xl = lib()
    g, u = _fields(32, 1, 1, 4400, np.complex64)
    U = to_dev(u, np.complex64)
    out = torch.empty_like(U)
    L = xl.load()
    gr = xl.Grid.of(g)
    z = (ctypes.c_double * 1)(100.0)
    # NULL save buffer
    st = L.xl_rs_propagate_save(U.data_ptr(), out.data_ptr(), None, 1, ctypes.byref(gr), LAM, z, 0,
                                xl.C64, None)
    assert st == xl.ERR_ARG
    # save buffer aliasing the output
    st = L.xl_rs_propagate_save(U.data_ptr(), out.data_ptr(), out.data_ptr(), 1, ctypes.byref(gr),
                                LAM, z, 0, xl.C64, None)
    assert st == xl.ERR_ARG
    # distance gradient without the saved transforms
    G = torch.empty_like(U)
    gz = torch.empty(1, dtype=torch.float64, device="cuda")
    st = L.xl_rs_propagate_backward_saved(G.data_ptr(), None, None, gz.data_ptr(), 1,
                                          ctypes.byref(gr), LAM, z, 0, xl.C64, None)
    assert st == xl.ERR_ARG


def test_autograd_uses_saved_spectra():
    """The autograd wrapper's distance gradient equals the explicit adjoint with u_in."""
    import torch
    xl = lib()
    from paper_2310_08408_gb300 import autograd
    g, u = _fields(64, 1, 2, 4500, np.complex64)
    U = to_dev(u, np.complex64)
    z = torch.tensor([600.0, 900.0], dtype=torch.float64, device="cuda", requires_grad=True)
    Ur = U.clone().requires_grad_(True)
    out = autograd.RSPropagate.apply(Ur, z, g, LAM, False)
    W = to_dev(inputs.random_unit(4501, (2, 64, 64)).astype(np.complex64), np.complex64)
    loss = (out * W.conj()).real.sum()
    loss.backward()
    gi, gz = xl.rs_propagate_backward(W, U, g, LAM, z.detach(), want_field=True, want_dz=True)
    assert torch.equal(Ur.grad, gi)
    assert torch.allclose(z.grad, gz, rtol=1e-5, atol=0)
