"""GPU: model checkpoint (mfa_model_get_ctrl, mfa_model_save, mfa_model_load).  A saved
and reloaded model holds bit-identical stored values and gives bit-identical decodes and
renders, for every storage type, non-uniform knots and mixed degrees, and for a model made
by the least-squares fit; the stored values are the input rounded once to the storage type;
the file has the documented size."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfa():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as m
    return m


def _renders_and_decodes(mfa, m):
    import torch
    cam = synth.camera_persp((1.7, 1.3, 2.2), (0.5, 0.5, 0.5), (0, 1, 0), 38.0)
    tf = mfa.transfer_fn(synth.ramp_tf(64, 0.1), shading=True)
    img = mfa.render(m, cam, tf, 40, 32, 96).cpu().numpy()
    pts = torch.rand((5000, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    v, g = mfa.decode(m, pts)
    return img, v.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("storage", [1, 2, 3])
def test_save_load_round_trip(mfa, orc, tmp_path, storage):
    rng = np.random.default_rng(40 + storage)
    degree, nctrl = (2, 3, 4), (13, 11, 12)
    knots = [synth.knots_nonuniform(nctrl[a], degree[a], rng) for a in range(3)]
    P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 5), knots, degree, rng, 0.01)
    m = mfa.Model(degree, nctrl, knots, P, storage=storage)
    stored = m.ctrl()
    expect = {1: np.asarray(P, np.float64).astype(np.float32), 2: orc.round_to_f16(P).astype(np.float16),
              3: None}[storage]
    if storage == 3:
        bits = stored.astype(np.uint32) << 16
        np.testing.assert_array_equal(bits.view(np.float32).astype(np.float64), orc.round_to_bf16(P))
    else:
        np.testing.assert_array_equal(stored, expect)
    path = os.path.join(tmp_path, f"m{storage}.mfa")
    m.save(path)
    nbytes = 64 + 8 * sum(nctrl[a] + degree[a] + 1 for a in range(3)) + int(np.prod(nctrl)) * (4 if storage == 1 else 2)
    assert os.path.getsize(path) == nbytes
    r = mfa.Model.load(path)
    assert r.degree == degree and r.nctrl == nctrl and r.storage == storage
    np.testing.assert_array_equal(r.ctrl().view(np.uint8), stored.view(np.uint8))
    assert r.info() == m.info()
    for a, b in zip(_renders_and_decodes(mfa, m), _renders_and_decodes(mfa, r)):
        np.testing.assert_array_equal(a, b)


def test_fitted_model_round_trip(mfa, tmp_path):
    data = synth.MarschnerLobb().grid_device(48)
    m, err = mfa.model_fit((3, 3, 3), (20, 20, 20), None, data)
    path = os.path.join(tmp_path, "fit.mfa")
    m.save(path)
    r = mfa.Model.load(path)
    assert r.info()["cardinal"] and r.info() == m.info()
    for a, b in zip(_renders_and_decodes(mfa, m), _renders_and_decodes(mfa, r)):
        np.testing.assert_array_equal(a, b)


def test_load_rejects_bad_files(mfa, tmp_path):
    m = mfa.Model((3, 3, 3), (8, 8, 8), None, np.zeros((8, 8, 8)))
    path = os.path.join(tmp_path, "ok.mfa")
    m.save(path)
    raw = open(path, "rb").read()
    for name, blob in (("short", raw[:40]), ("magic", b"XX" + raw[2:]), ("trunc", raw[:-3]), ("extra", raw + b"\0")):
        bad = os.path.join(tmp_path, name + ".mfa")
        open(bad, "wb").write(blob)
        with pytest.raises(mfa.MfaError):
            mfa.Model.load(bad)
    with pytest.raises(mfa.MfaError):
        m.save(os.path.join(tmp_path, "no_such_dir", "x.mfa"))
