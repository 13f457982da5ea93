"""GPU parity of the beam splitter and its adjoint against the FP64 oracle (element by element
on the same seeded inputs), null ports, in-place use, and the autograd wrapper."""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C128, TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu
RS = [0.2, 0.5, 0.93]


def _fields(seed, dtype, shape=(3, 2, 48, 40)):
    a = (inputs.random_unit(seed, shape)).astype(dtype)
    b = (inputs.random_unit(seed + 1, shape)).astype(dtype)
    return a, b


@pytest.mark.parametrize("dtype,tol", [(np.complex64, TOL_C64), (np.complex128, TOL_C128)])
def test_forward_and_adjoint(dtype, tol):
    import torch
    xl = lib()
    a, b = _fields(5200, dtype)
    gt, gr = _fields(5210, dtype)
    R = torch.tensor(RS, dtype=torch.float64, device="cuda")
    A, Bf, GT, GR = (to_dev(x, dtype) for x in (a, b, gt, gr))
    ot, orr = xl.beam_splitter(A, Bf, R)
    ga, gb, gR = xl.beam_splitter_backward(GT, GR, A, Bf, R)
    for e, Re in enumerate(RS):
        rt, rr = oracle.beam_splitter(a[e].astype(np.complex128), b[e].astype(np.complex128), Re)
        assert rel(to_np(ot)[e], rt) < tol and rel(to_np(orr)[e], rr) < tol
        qa, qb, qR = oracle.beam_splitter_backward(gt[e].astype(np.complex128), gr[e].astype(np.complex128),
                                                   a[e].astype(np.complex128), b[e].astype(np.complex128), Re)
        assert rel(to_np(ga)[e], qa) < tol and rel(to_np(gb)[e], qb) < tol
        assert abs(to_np(gR)[e] - qR) < (1e-5 if dtype == np.complex64 else 1e-10) * max(1.0, abs(qR))


def test_null_ports_and_in_place():
    import torch
    xl = lib()
    a, b = _fields(5220, np.complex64)
    R = torch.tensor(RS, dtype=torch.float64, device="cuda")
    A, Bf = to_dev(a, np.complex64), to_dev(b, np.complex64)
    # a single beam entering port a
    ot, orr = xl.beam_splitter(A, None, R)
    for e, Re in enumerate(RS):
        rt, rr = oracle.beam_splitter(a[e].astype(np.complex128), None, Re)
        assert rel(to_np(ot)[e], rt) < TOL_C64 and rel(to_np(orr)[e], rr) < TOL_C64
    # in place: outputs over the inputs
    ref_t, ref_r = xl.beam_splitter(A, Bf, R)
    A2, B2 = A.clone(), Bf.clone()
    xl.beam_splitter(A2, B2, R, out_t=A2, out_r=B2)
    assert torch.equal(A2, ref_t) and torch.equal(B2, ref_r)
    # zero cotangent on one port
    ga, gb, gR = xl.beam_splitter_backward(None, Bf, A, Bf, R)
    for e, Re in enumerate(RS):
        qa, qb, qR = oracle.beam_splitter_backward(None, b[e].astype(np.complex128),
                                                   a[e].astype(np.complex128), b[e].astype(np.complex128), Re)
        assert rel(to_np(ga)[e], qa) < TOL_C64 and rel(to_np(gb)[e], qb) < TOL_C64
        assert abs(to_np(gR)[e] - qR) < 1e-5 * max(1.0, abs(qR))


def test_autograd_interferometer():
    """Mach-Zehnder with a phase mask in one arm: autograd through two splitters gives the
    gradients of the explicit adjoint chain, and the balanced case sends all light to port r."""
    import torch
    xl = lib()
    from paper_2310_08408_gb300.autograd import BeamSplitter
    a, _ = _fields(5230, np.complex64, (2, 32, 32))
    A = to_dev(a, np.complex64)
    zero = torch.zeros_like(A)
    R1 = torch.tensor([0.5, 0.3], dtype=torch.float64, device="cuda", requires_grad=True)
    R2 = torch.tensor([0.5, 0.6], dtype=torch.float64, device="cuda", requires_grad=True)
    phi = torch.zeros((2, 32, 32), dtype=torch.float32, device="cuda", requires_grad=True)
    u1, u2 = BeamSplitter.apply(A, zero, R1)
    u1 = u1 * torch.exp(1j * phi)
    ot, orr = BeamSplitter.apply(u1, u2, R2)
    # element 0 is balanced: dark transmitted port
    assert float(ot[0].detach().abs().max()) < 1e-6
    loss = (ot.abs() ** 2).sum()
    loss.backward()
    # explicit chain
    with torch.no_grad():
        v1, v2 = xl.beam_splitter(A, None, R1.detach())
        w1 = v1 * torch.exp(1j * phi.detach())
        t2, r2 = xl.beam_splitter(w1, v2, R2.detach())
        g1, g2, gR2 = xl.beam_splitter_backward(2 * t2, None, w1, v2, R2.detach())
        gphi = (g1 * torch.conj(w1)).imag
        gw1 = g1 * torch.exp(-1j * phi.detach())
        _, _, gR1 = xl.beam_splitter_backward(gw1, g2, A, None, R1.detach())
    assert torch.allclose(R2.grad, gR2, rtol=1e-6, atol=1e-6)
    assert torch.allclose(R1.grad, gR1, rtol=1e-6, atol=1e-6)
    assert torch.allclose(phi.grad, gphi.float(), rtol=1e-5, atol=1e-5)
