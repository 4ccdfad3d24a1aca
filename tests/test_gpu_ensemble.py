"""The 64-box ensemble (numpy default_rng(0) draws: 48^3 to 192x128x128 boxes
with one or two swimmers, drive period 2000 steps) stepped as one autotuned
batch, as the benchmark steps it, against FP64 oracle runs of four sampled
boxes, one of each size class, over one drive period
(tests/golden/ensemble_samples.json, written by make_ensemble_golden.py from
oracle/ alone).

Checked for each sampled box: x_cm of every swimmer every 100 steps (Sec. 3,
Eq. vel_swim) within 1e-3 of the distance travelled, the mean swimming
velocity over the period within 1 %, and the velocity u at the stored cells
(2048 random ones and the 512 of largest |u|) after the period as a relative
L2 error over that sample, <= 1e-5 (FP32 storage)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_ensemble_sampled_boxes_against_oracle(gpu_lib):
    import torch
    from paper_2202_12147_gb300.ensemble import EnsembleShare
    from workloads import assemble, ensemble_boxes
    path = os.path.join(HERE, "golden", "ensemble_samples.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle runs of the ensemble")
    with open(path) as fh:
        gold = json.load(fh)
    steps, every = gold["steps"], gold["every"]
    boxes = ensemble_boxes()
    share = EnsembleShare(boxes, [assemble(b) for b in boxes], 0, 1)
    sampled = {int(k): v for k, v in gold["boxes"].items()}
    for k, g in sampled.items():
        assert list(boxes[k].dims) == g["dims"] and len(boxes[k].swimmers) == g["n_swimmers"]
    sims = {k: share.sims[share.mine.index(k)] for k in sampled}

    def x_cm(k):
        return [sims[k].swimmer_state(s)["x_cm"] for s in range(sims[k].n_swimmers)]

    xs = {k: [x_cm(k)] for k in sampled}
    rep = share.autotune(steps_per_trial=2)
    done = rep["steps_taken"]
    assert 0 < done < every
    share.lb_step(every - done)
    done = every
    for k in sampled:
        xs[k].append(x_cm(k))
    while done < steps:
        share.lb_step(every)
        done += every
        for k in sampled:
            xs[k].append(x_cm(k))
    for k, g in sampled.items():
        xg = np.array(xs[k])
        xo = np.array([x for _, x in g["x_cm"]])
        assert xg.shape == xo.shape
        travel = np.abs(xo - xo[0]).max()
        x_err = np.abs(xg - xo).max() / travel
        vg = (xg[-1, :, 0] - xg[0, :, 0]) / steps
        vo = (xo[-1, :, 0] - xo[0, :, 0]) / steps
        v_err = np.abs(vg - vo).max() / np.abs(vo).min()
        _, u = sims[k].lb_get_macros()
        cells = g["u_sample"]["cells"]
        idx = torch.tensor(cells, dtype=torch.long, device=u.device)
        ug = u[idx].cpu().numpy().astype(np.float64)
        uo = np.array(g["u_sample"]["u"])
        u_err = np.linalg.norm(ug - uo) / np.linalg.norm(uo)
        print(f"box {k} {tuple(g['dims'])}: x_cm {x_err:.2e} of the travel, period velocity {v_err:.2e}, "
              f"velocity sample rel. L2 {u_err:.2e}")
        assert x_err < 1e-3
        assert v_err < 1e-2
        assert u_err < 1e-5
    share.close()
