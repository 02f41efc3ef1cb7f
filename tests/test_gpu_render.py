"""GPU parity of the particle renderer (App. D.2 screen-space splatting) against the FP64 oracle on the
same FP32 camera and positions: the splatted depth, the distance-scaled bilateral filter, the normals
and the Lambert colour, pixel by pixel.

Pixels where the oracle finds a coverage test within 1e-4 of flipping (with the particle in front),
and for the later steps the pixels within reach of those (the filter window, the differences), are
excluded; so are pixels whose difference side is within 1e-5 of switching. There must be few."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_04659_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_04659_gb300 import build
    build.build()
    yield


def _setup(W=320, H=256, K=4, fov=40.0, eye=(0.55, 0.55, -0.35), target=(0.5, 0.2, 0.5), radius=0.004):
    from paper_2302_04659_gb300.render import Camera, Style
    cam = Camera.looking(W, H, fov, eye, target)
    style = Style(radius=radius, smooth=0.008, sigma_depth=0.01, window=K)
    # the oracle gets the FP32 values the library sees, widened
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ocam = oracle.Camera(W, H, float(np.float32(cam.fx)), float(np.float32(cam.fy)), float(np.float32(cam.cx)),
                         float(np.float32(cam.cy)), tuple(f32(cam.eye)), f32(cam.rot), float(np.float32(cam.near_z)))
    ors = oracle.RenderParams(float(np.float32(style.radius)), float(np.float32(style.smooth)),
                              float(np.float32(style.sigma_depth)), K, tuple(f32(style.light)), tuple(f32(style.albedo)),
                              float(np.float32(style.ambient)), tuple(f32(style.background)))
    return cam, style, ocam, ors


def _dilate(mask, r):
    out = mask.copy()
    H, W = mask.shape
    for dj in range(-r, r + 1):
        for di in range(-r, r + 1):
            sh = np.zeros_like(mask)
            sh[max(dj, 0):H + min(dj, 0), max(di, 0):W + min(di, 0)] = mask[max(-dj, 0):H + min(-dj, 0),
                                                                          max(-di, 0):W + min(-di, 0)]
            out |= sh
    return out


def test_render_matches_oracle_pinch():
    from paper_2302_04659_gb300.render import Renderer
    sc = scenes.pinch_scene(seed=1000, N=200_000)
    cam, style, ocam, ors = _setup()
    r = Renderer(cam, style)
    x = torch.from_numpy(sc.x).cuda()
    r.render(x)
    torch.cuda.synchronize()
    depth, smooth, normal, rgb = (t.cpu().numpy().astype(np.float64) for t in (r.depth, r.smooth, r.normal, r.rgb))
    od, amb, drawn = oracle.splat_depth(ocam, ors, sc.x.astype(np.float64))
    assert drawn == sc.N
    K = ors.window
    fin = np.isfinite(od)
    assert fin.sum() > 0.1 * od.size, "the body should fill a good part of the image"
    assert amb.sum() <= 2e-3 * od.size
    # step 1: coverage exact and depth to FP32 rounding away from ambiguous pixels
    ok = ~amb
    assert np.array_equal(np.isfinite(depth)[ok], fin[ok])
    both = ok & fin
    # z - r sqrt(1 - s^2): FP32 evaluates s^2 to ~2e-5 (pixel coordinates of a few hundred, footprints of
    # ~1.5 px), and d sqrt(1 - s^2) / d s^2 = 1 / (2 sqrt(1 - s^2)) reaches 50 where 1 - s^2 = 1e-4 (the
    # edge of the non-ambiguous band): |dz| <= r * 2e-5 * 50 = 1e-3 r there, FP32 rounding elsewhere
    err = np.abs(depth[both] - od[both])
    assert err.max() <= 1e-3 * ors.radius
    assert np.quantile(err, 0.999) <= 1e-6 * od[both].max()
    # step 2
    osm = oracle.bilateral(ocam, ors, od)
    ok2 = ~_dilate(amb, K) & fin
    assert ok2.sum() > 0.9 * fin.sum()
    assert np.abs(smooth[ok2] - osm[ok2]).max() <= 1e-5 * osm[ok2].max()
    assert np.all(np.isinf(smooth[~fin & ~_dilate(amb, K)]))
    # steps 3 and 4
    on, orgb, amb3 = oracle.shade(ocam, ors, osm)
    ok3 = ~_dilate(amb, K + 1) & ~amb3
    assert ok3.sum() > 0.9 * od.size
    assert np.abs(normal[ok3] - on[ok3]).max() <= 2e-3
    assert np.abs(rgb[ok3] - orgb[ok3]).max() <= 2e-3
    # most pixels agree far more tightly than the bound
    assert np.median(np.abs(normal[ok3 & fin] - on[ok3 & fin])) <= 1e-4


def test_render_sim_in_place_equals_render_of_read_state():
    """The handle's particles rendered where the simulation keeps them (sorted order, no copy) give the
    same images as rendering the positions read back in the caller's order."""
    from gpu_helpers import make_sim
    from paper_2302_04659_gb300.render import Renderer
    sc = scenes.pinch_scene(seed=1001, N=100_000)
    sim = make_sim(sc)
    sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    sim.set_shapes(sc.shapes)
    sim.set_colliders(*scenes.finger_state(sc, 0.1))
    sim.substep(25)
    cam, style, _, _ = _setup()
    a = Renderer(cam, style)
    b = Renderer(cam, style)
    a.render_sim(sim)
    b.render(sim.read_state(on_device=True)["x"])
    torch.cuda.synchronize()
    for name in ("depth", "smooth", "normal", "rgb"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    sim.close()


def test_render_edge_cases():
    from paper_2302_04659_gb300 import _native as mpm
    from paper_2302_04659_gb300.render import Renderer, Style
    cam, style, ocam, ors = _setup(W=64, H=48, radius=0.02)
    r = Renderer(cam, style)
    # nothing to draw: background everywhere
    r.render(torch.zeros((3, 0), device="cuda"))
    torch.cuda.synchronize()
    assert torch.isinf(r.depth).all()
    assert torch.equal(r.rgb, torch.zeros_like(r.rgb))
    # three particles (columns): behind the camera, in front but off screen, in view
    x = torch.tensor([[0.55, 5.0, 0.5], [0.55, 0.5, 0.3], [-1.0, 0.5, 0.4]], device="cuda")
    r.render(x)
    torch.cuda.synchronize()
    od, amb, drawn = oracle.splat_depth(ocam, ors, x.cpu().numpy().astype(np.float64))
    assert drawn == 2
    fin = np.isfinite(od)
    assert 0 < fin.sum() < 40
    assert np.array_equal(torch.isfinite(r.depth).cpu().numpy()[~amb], fin[~amb])
    # window 0: the smoothed depth is the splatted one
    r0 = Renderer(cam, Style(radius=0.05, smooth=0.01, sigma_depth=0.01, window=0))
    sc = scenes.cube_scene("floor")
    r0.render(torch.from_numpy(sc.x).cuda())
    torch.cuda.synchronize()
    assert torch.equal(r0.depth, r0.smooth)
    # invalid arguments are refused before anything is enqueued
    bad = Style(radius=-1.0, smooth=0.01, sigma_depth=0.01)
    with pytest.raises(mpm.MpmError):
        Renderer(cam, bad).render(x)
    with pytest.raises(mpm.MpmError):
        mpm.mpm_render(cam.c(), style.c(), 3, 3, x.data_ptr(), 0, 0, 0, r.rgb.data_ptr(), r.ws.data_ptr(), 16)
