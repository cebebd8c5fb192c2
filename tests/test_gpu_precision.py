"""GPU: the precision sweep at full size -- degree 3, 512x512x256 control points,
non-uniform knots (spacings 1:4), turbulence field; FP32, FP16 and BF16 storage.

For each storage type the KERNEL error (GPU against the FP64 oracle run on the same
rounded control points) must meet the FP32 gates; the TOTAL error (against the FP64
control points) is measured and printed.  Decode: 2^22 uniform points, every one checked.
Render: 2048^2 with 2048 samples per ray, Phong; 8192 seeded pixels plus two full rows
through the oracle.
"""
import numpy as np
import pytest

import synth
from metrics import GRAD_TOL, IMAGE_RMSE_TOL, VALUE_TOL, grad_error, image_rmse, value_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    return synth.config3(dtype_in=np.float64)


@pytest.mark.parametrize("storage,name", [(1, "f32"), (2, "f16"), (3, "bf16")])
def test_precision_sweep_full_size(orc, workload, storage, name):
    import torch
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as mfa
    spec, job = workload.model, workload.render
    P = spec.ctrl64
    stored = {1: lambda x: x.astype(np.float32).astype(np.float64), 2: orc.round_to_f16, 3: orc.round_to_bf16}[storage](P)
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, P, storage=storage)
    kern = orc.Model(spec.degree, spec.nctrl, spec.knots, stored)
    exact = orc.Model(spec.degree, spec.nctrl, spec.knots, P)

    pts = workload.decode_points
    val, grad = mfa.decode(model, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    v, g = val.cpu().numpy(), grad.cpu().numpy()
    vk, gk = kern.decode(pts)
    ve, ge = exact.decode(pts)
    ev_k, eg_k = value_error(v, vk, stored), grad_error(g, gk)
    ev_t, eg_t = value_error(v, ve, P), grad_error(g, ge)

    W, H = job.width, job.height
    info = model.info()
    vmin, vmax = info["vmin"], info["vmax"]
    tf = mfa.transfer_fn(job.tf, shading=True, vmin=vmin, vmax=vmax)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img = mfa.render(model, job.camera, tf, W, H, job.n_samples, samples_out=cnt)
    torch.cuda.synchronize()
    rng = np.random.default_rng(31)
    pix = np.concatenate([rng.choice(W * H, 8192, replace=False), np.arange(700 * W, 701 * W),
                          np.arange(1400 * W, 1401 * W)])
    gimg = img.cpu().numpy().reshape(-1, 4)[pix]
    rk, _ = orc.render(kern, job.camera, job.tf, W, H, job.n_samples, shading=True, vmin=vmin, vmax=vmax, pixels=pix)
    rt, _ = orc.render(exact, job.camera, job.tf, W, H, job.n_samples, shading=True, vmin=vmin, vmax=vmax, pixels=pix)
    rmse_k, rmse_t = image_rmse(gimg, rk), image_rmse(gimg, rt)
    print(f"{name}: kernel e_v={ev_k:.2e} e_g={eg_k:.2e} rmse={rmse_k.max():.2e} | "
          f"total e_v={ev_t:.2e} e_g={eg_t:.2e} rmse={rmse_t.max():.2e} | samples={int(cnt.item())}")
    assert ev_k <= VALUE_TOL and eg_k <= GRAD_TOL
    assert np.all(rmse_k <= IMAGE_RMSE_TOL)
    assert rk[:, 3].max() > 0.1
