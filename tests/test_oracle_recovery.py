"""Recovery of a seeded ground truth on a tiny grid (Sec. 5.1: pixel and volume
errors fall as iterations proceed; Sec. 5.2: more cameras give lower error).
These pins are qualitative, as the paper's own statements are."""
import numpy as np

from paper_1809_06417_gb300 import synth


def _setup(orc, n=12, views=8, side=32, seed=1):
    shape, origin, h = synth.unit_grid(n)
    cams = synth.ring_cameras(views, side, side, elevation_jitter_deg=10.0, seed=seed)
    sc = orc.Scene(shape, origin, h, cams)
    gt = synth.blobs_volume(n, seed, radius_range=(1.5, 3.0))
    P = orc.make_params(step=0.5)
    img, _ = orc.render(sc, gt, P)
    gt[..., :3] /= img.max()
    img /= img.max()
    targets, mask, bbox = orc.prepare_targets(img, 30 / 255)
    return sc, gt, targets, mask, bbox


def test_errors_fall_with_iterations(orc):
    sc, gt, targets, mask, bbox = _setup(orc)
    P = orc.make_params(step=0.5, alpha_l=0.005)
    v0 = gt.copy()
    v0[..., :3] = 0.0  # the volume starts at zero (Sec. 3)
    vols, rm = [], []
    v = v0
    for it in range(6):
        v, rmse, _ = orc.reconstruct(sc, v, P, targets, mask, bbox, 5, first_iteration=5 * it)
        rm.extend(rmse[:, 1])
        vols.append(np.sqrt(np.mean((v[..., :3] - gt[..., :3]) ** 2)))
    rm = np.array(rm)
    vol0 = np.sqrt(np.mean(gt[..., :3] ** 2))
    assert np.all(np.diff(rm[:10]) < 0)           # pixel error falls at first
    assert rm[-1] < 0.2 * rm[0]
    assert vols[-1] < 0.7 * vol0                  # the volume moves toward the truth
    assert vols[-1] < vols[0]


def test_more_cameras_lower_volume_error(orc):
    errs = []
    for views in (2, 8):
        sc, gt, targets, mask, bbox = _setup(orc, views=views)
        P = orc.make_params(step=0.5, alpha_l=0.005 * 8 / views)
        v0 = gt.copy()
        v0[..., :3] = 0.0
        v, _, _ = orc.reconstruct(sc, v0, P, targets, mask, bbox, 30)
        errs.append(np.sqrt(np.mean((v[..., :3] - gt[..., :3]) ** 2)))
    assert errs[1] < errs[0]
