"""GPU optical table (autograd over the C ABI) against the oracle's table and its adjoint
gradients (which the CPU tests pin by float64 central finite differences).

Table (Results / Methods: virtual optical tables): x-polarised Gaussian -> SLM1 -> RS z1 -> SLM2
-> half-wave plate (theta) -> VRS z2 -> lens f -> VCZT f onto the camera window -> second-moment
spot size of the total intensity. Gradients for both masks, theta, z1 and z2.
"""
import numpy as np
import pytest

import oracle
import oracle.table as otable
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_LOSS, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def _run(n, pitch, lam, w0, z1, z2, theta, f, m, width, seed, dtype, rdtype, checkpoint=False):
    import torch
    lib()
    from paper_2310_08408_gb300 import table
    g = inputs.Grid.centred(n, pitch)
    win = inputs.Window.centred(m, width)
    src = inputs.x_polarised_gaussian(g, w0)
    phi1 = inputs.random_phase(g, seed)
    phi2 = inputs.random_phase(g, seed + 1)
    geo = table.TableGeometry(g.astuple(), win.astuple(), lam, f)
    P1 = to_dev(phi1[None].astype(rdtype), rdtype).requires_grad_(True)
    P2 = to_dev(phi2[None].astype(rdtype), rdtype).requires_grad_(True)
    th = torch.tensor([theta], dtype=torch.float64, device="cuda", requires_grad=True)
    Z1 = torch.tensor([z1], dtype=torch.float64, device="cuda", requires_grad=True)
    Z2 = torch.tensor([z2], dtype=torch.float64, device="cuda", requires_grad=True)
    S = to_dev(src[None, None].astype(dtype), dtype)
    loss = table.table_loss(geo, S, P1, P2, th, Z1, Z2, checkpoint=checkpoint)
    loss.sum().backward()
    # oracle on the same rounded inputs
    t = otable.Table(g.astuple(), win.astuple(), lam, f)
    s64 = src.astype(dtype).astype(np.complex128)
    p1 = phi1.astype(rdtype).astype(np.float64)
    p2 = phi2.astype(rdtype).astype(np.float64)
    L, planes = otable.forward(t, s64, p1, p2, theta, z1, z2)
    gr = otable.backward(t, s64, p1, p2, theta, z1, z2, planes)
    return (float(to_np(loss)[0]), L, to_np(P1.grad)[0], gr["phi1"], to_np(P2.grad)[0], gr["phi2"],
            float(to_np(th.grad)[0]), gr["theta"], float(to_np(Z1.grad)[0]), gr["z1"],
            float(to_np(Z2.grad)[0]), gr["z2"])


@pytest.mark.parametrize("checkpoint", [False, True])
@pytest.mark.parametrize("dtype,rdtype,tl,tg", [(np.complex64, np.float32, TOL_LOSS, 1e-3),
                                                (np.complex128, np.float64, 1e-10, 1e-8)])
def test_table_small(dtype, rdtype, tl, tg, checkpoint):
    """Both ways of keeping what the distance gradients need: input spectra, or the plane fields
    with the spectra recomputed in the adjoints (checkpoint)."""
    r = _run(64, 1.0, 0.6328, 12.0, 300.0, 250.0, 0.3, 800.0, 40, 48.0, 31, dtype, rdtype, checkpoint)
    Lg, Lo, g1, o1, g2, o2, gt, ot, gz1, oz1, gz2, oz2 = r
    assert abs(Lg - Lo) / abs(Lo) < tl
    assert rel(g1, o1) < tg and rel(g2, o2) < tg
    for a, b in ((gt, ot), (gz1, oz1), (gz2, oz2)):
        assert abs(a - b) / abs(b) < tg


def test_table_config_1024():
    """The optical-table workload at its full size: 1024^2 at 1 um, lambda 0.6328 um, w0 200 um,
    z1 = z2 = 20 mm, theta 0.3, f = 5 mm, camera 256^2 over 64 um."""
    w = inputs.WORKLOADS["table1024"]
    r = _run(w["n"], w["pitch"], w["wavelength"], w["w0"], w["z1"], w["z2"], w["theta"], w["f"],
             w["window_m"], w["window_w"], w["seed"], np.complex64, np.float32)
    Lg, Lo, g1, o1, g2, o2, gt, ot, gz1, oz1, gz2, oz2 = r
    assert abs(Lg - Lo) / abs(Lo) < TOL_LOSS
    assert rel(g1, o1) < 1e-3 and rel(g2, o2) < 1e-3
    errs = [abs(a - b) / abs(b) for a, b in ((gt, ot), (gz1, oz1), (gz2, oz2))]
    assert max(errs) < 1e-3, errs
