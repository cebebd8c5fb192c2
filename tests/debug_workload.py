"""Runs a spread of workloads through the library named by MFA_LIB (the debug build in
tests/test_gpu_debug.py) and prints its debug status as one JSON line: every kernel family
(render variants 1-7, segments, isosurfaces, decode, batches, fits, the ground-truth render
and metrics), uniform and non-uniform knots, degrees 1-4, all storage types, points
outside the box."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2312_15073_gb300 as mfa  # noqa: E402
import synth  # noqa: E402


def main():
    rng = np.random.default_rng(77)
    cam = synth.camera_persp((1.7, 1.3, 2.2), (0.5, 0.5, 0.5), (0, 1, 0), 40.0)
    tf = mfa.transfer_fn(synth.ramp_tf(64, 0.1), shading=True)
    pts = torch.from_numpy(rng.uniform(-0.1, 1.1, (20000, 3)).astype(np.float32)).cuda()
    models = []
    for degree, nctrl, uniform, storage in (((3, 3, 3), (20, 18, 22), True, 1), ((3, 3, 3), (19, 17, 21), False, 2),
                                            ((2, 3, 4), (12, 14, 11), False, 1), ((1, 1, 1), (9, 8, 7), True, 3),
                                            ((4, 4, 4), (13, 12, 14), True, 1), ((2, 2, 2), (16, 15, 17), True, 2)):
        knots = [synth.knots_uniform(nctrl[a], degree[a]) if uniform else synth.knots_nonuniform(nctrl[a], degree[a], rng)
                 for a in range(3)]
        P = synth.sample_ctrl(synth.GaussianSum.draw(rng, 5), knots, degree, rng, 0.01)
        m = mfa.Model(degree, nctrl, knots, P, storage=storage)
        models.append(m)
        mfa.decode(m, pts)
        mfa.decode(m, pts, want_grad=False)
        for variant in range(0, 8):   # 6 and 7 fall back to 4 on non-cardinal models
            mfa.render(m, cam, tf, 33, 27, 80, variant=variant)
        clear_low = synth.ramp_tf(64, 0.1).copy()
        clear_low[:32, 3] = 0.0
        mfa.render(m, cam, mfa.transfer_fn(clear_low, shading=True), 33, 27, 80, variant=7)
        mfa.render_segments(m, cam, tf, 33, 27, 80, (2, 2, 2))
        mfa.render_iso(m, cam, tf, 33, 27, 80, float(np.median(P)))
    reqs = [mfa.Request(m, cam, tf, 24, 20, 64) for m in models]
    mfa.render_batch(reqs)
    data = synth.MarschnerLobb().grid_device(40)
    fitted, _ = mfa.model_fit((2, 2, 2), (16, 16, 16), None, data)
    encoded, _ = mfa.model_encode((3, 3, 3), data, 1e-2, max_ctrl=(20, 20, 20))
    truth = mfa.render_ml(cam, tf, 33, 27, 80)
    mfa.image_compare(mfa.render(fitted, cam, tf, 33, 27, 80), truth)
    torch.cuda.synchronize()
    print(json.dumps(mfa.debug_status()))


if __name__ == "__main__":
    main()
