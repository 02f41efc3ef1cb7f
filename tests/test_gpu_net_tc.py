"""GPU parity of the tensor-core (tcgen05) forward convolution with the FP64 network oracle, on the
surrogate's layer shapes and ragged boxes; masked (tiled) outputs against unmasked ones; the kernel's
bounded-wait error word stays clear."""
import numpy as np
import pytest
import torch

from oracle import net_oracle as no

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(303)


@pytest.fixture(scope="module")
def mpm():
    from paper_2302_04659_gb300 import _native, build
    build.build()
    return _native


def packed(mpm, w, cin, cout):
    out = torch.zeros(mpm.mpm_conv3d_tc_packed_bytes(cin, cout), dtype=torch.uint8, device="cuda")
    mpm.mpm_conv3d_pack_tc(cin, cout, w.data_ptr(), out.data_ptr())
    return out


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


CASES = [((1, 16, 8), 32, 32), ((2, 19, 11), 32, 32), ((3, 17, 9), 4, 32), ((5, 21, 13), 32, 3),
         ((2, 18, 10), 16, 16), ((4, 5, 3), 32, 32), ((1, 1, 1), 4, 32)]


@pytest.mark.parametrize("box,cin,cout", CASES + [((64, 64, 64), 32, 32)])  # the last: a full 64^3 grid
@pytest.mark.parametrize("relu,y_f32", [(0, 1), (1, 0)])
def test_tc_forward_matches_oracle(mpm, box, cin, cout, relu, y_f32):
    x = torch.from_numpy(RNG.normal(size=box + (cin,)).astype(np.float32)).to(torch.bfloat16).cuda()
    w = torch.from_numpy((0.2 * RNG.normal(size=(27, cout, cin))).astype(np.float32)).to(torch.bfloat16).cuda()
    b = torch.from_numpy(RNG.normal(size=cout).astype(np.float32)).cuda()
    y = torch.zeros(box + (cout,), dtype=torch.float32 if y_f32 else torch.bfloat16, device="cuda")
    wp = packed(mpm, w, cin, cout)
    mpm.mpm_conv3d_forward_tc(*box, cin, cout, x.data_ptr(), wp.data_ptr(), b.data_ptr(), relu, y_f32, y.data_ptr())
    assert mpm.mpm_net_tc_status(clear=1) == 0
    ref = no.conv3d_forward(x.float().cpu().numpy(), w.float().cpu().numpy(), b.cpu().numpy())
    if relu:
        ref = no.relu(ref)
    got = y.float().cpu().numpy()
    # FP32 output: BF16 products are exact, only the FP32 accumulation order differs
    assert rel(got, ref) <= (1e-5 if y_f32 else 1e-2)


def test_tc_masked_tiles_match_unmasked_on_the_mask(mpm):
    box, cin, cout = (6, 40, 24), 32, 32
    x = torch.from_numpy(RNG.normal(size=box + (cin,)).astype(np.float32)).to(torch.bfloat16).cuda()
    w = torch.from_numpy((0.2 * RNG.normal(size=(27, cout, cin))).astype(np.float32)).to(torch.bfloat16).cuda()
    wp = packed(mpm, w, cin, cout)
    mask = np.zeros(box, np.uint8)
    mask[2:4, 5:9, 3:6] = 1
    md = torch.from_numpy(mask).cuda()
    ntiles = mpm.mpm_conv3d_tc_tile_count(*box)
    assert ntiles == 6 * 3 * 3
    dist = torch.zeros(ntiles, dtype=torch.uint8, device="cuda")
    mpm.mpm_conv3d_tc_tile_dist(*box, md.data_ptr(), dist.data_ptr())
    full = torch.zeros(box + (cout,), dtype=torch.float32, device="cuda")
    part = torch.full(box + (cout,), 7.0, dtype=torch.float32, device="cuda")
    mpm.mpm_conv3d_forward_tc(*box, cin, cout, x.data_ptr(), wp.data_ptr(), 0, 0, 1, full.data_ptr())
    mpm.mpm_conv3d_forward_tc(*box, cin, cout, x.data_ptr(), wp.data_ptr(), 0, 0, 1, part.data_ptr(), dist.data_ptr(), 2)
    assert mpm.mpm_net_tc_status(clear=1) == 0
    f, p = full.cpu().numpy(), part.cpu().numpy()
    # the distance map against a brute-force one
    d = dist.cpu().numpy()
    pts = np.argwhere(mask)
    for t in range(ntiles):
        x0, y0, z0 = (t % 3) * 8, ((t // 3) % 3) * 16, t // 9
        zs, ys, xs = [z0], range(y0, min(y0 + 16, box[1])), range(x0, min(x0 + 8, box[2]))
        best = 5
        for z in zs:
            for yy in ys:
                for xx in xs:
                    best = min(best, int(np.abs(pts - [z, yy, xx]).max(axis=1).min()))
        assert d[t] == min(best, 5), (t, d[t], best)
    # every voxel within distance 2 of the mask is computed exactly as without the mask
    near = np.zeros(box, bool)
    for z, yy, xx in pts:
        near[max(z - 2, 0):z + 3, max(yy - 2, 0):yy + 3, max(xx - 2, 0):xx + 3] = True
    np.testing.assert_array_equal(p[near], f[near])
    # tiles far from the mask are zero-filled, not left stale
    assert not (p == 7.0).any()
    assert (p == 0.0).any()


BACK_CASES = [((2, 19, 11), 32, 32), ((5, 21, 13), 32, 3), ((3, 17, 9), 4, 32), ((1, 1, 1), 32, 32),
              ((4, 16, 8), 16, 32)]


@pytest.mark.parametrize("box,cin,cout", BACK_CASES)
@pytest.mark.parametrize("masked", [0, 1])
def test_tc_backward_data_matches_oracle(mpm, box, cin, cout, masked):
    """The input gradient on the tensor cores (the forward kernel on the mirrored, channel-swapped weights,
    ReLU mask of the layer's input applied in the epilogue) against the oracle's adjoint on the same
    BF16 operands, and against the mma.sync input gradient."""
    nvox = int(np.prod(box))
    cp = 4 if cout <= 4 else (16 if cout <= 16 else 32)
    dy = torch.from_numpy(RNG.normal(size=box + (cout,)).astype(np.float32)).to(torch.bfloat16).cuda()
    w = torch.from_numpy((0.2 * RNG.normal(size=(27, cout, cin))).astype(np.float32)).to(torch.bfloat16).cuda()
    act = torch.from_numpy(RNG.normal(size=box + (cin,)).astype(np.float32)).to(torch.bfloat16).cuda()
    dyp = torch.empty(box + (cp,), dtype=torch.bfloat16, device="cuda")
    mpm.mpm_pad_channels_bf16(nvox, cout, cp, dy.data_ptr(), dyp.data_ptr())
    wa = torch.zeros(mpm.mpm_conv3d_tc_adjoint_packed_bytes(cin, cout), dtype=torch.uint8, device="cuda")
    mpm.mpm_conv3d_pack_tc_adjoint(cin, cout, w.data_ptr(), wa.data_ptr())
    dx = torch.zeros(box + (cin,), dtype=torch.bfloat16, device="cuda")
    mpm.mpm_conv3d_backward_data_tc(*box, cin, cout, dyp.data_ptr(), wa.data_ptr(),
                                    act.data_ptr() if masked else 0, dx.data_ptr())
    assert mpm.mpm_net_tc_status(clear=1) == 0
    assert torch.equal(dyp[..., :cout], dy) and (cp == cout or bool((dyp[..., cout:] == 0).all()))
    ref = no.conv3d_backward_data(dy.float().cpu().numpy(), w.float().cpu().numpy())
    if masked:
        ref = ref * (act.float().cpu().numpy() > 0)
    got = dx.float().cpu().numpy()
    assert rel(got, ref) <= 1e-2
    if masked:
        assert np.all(got[act.float().cpu().numpy() <= 0] == 0.0)
    # the mma.sync kernel of the same gradient
    dx2 = torch.zeros(box + (cin,), dtype=torch.bfloat16, device="cuda")
    mpm.mpm_conv3d_backward_data(mpm.MPM_NET_BF16, *box, cin, cout, dy.data_ptr(), w.data_ptr(),
                                 act.data_ptr() if masked else 0, dx2.data_ptr())
    assert rel(got, dx2.float().cpu().numpy()) <= 1e-2


# the last box is a full 64^3 grid: about 13 tiles per CTA accumulate in tensor memory (measured dW
# relative error 1.7e-6 there, 1e-7 to 3e-7 on the smaller boxes: longer FP32 sums)
WG_CASES = CASES + [((40, 33, 17), 32, 32), ((9, 38, 40), 4, 32), ((7, 37, 23), 32, 3), ((64, 64, 64), 32, 32)]


@pytest.mark.parametrize("box,cin,cout", WG_CASES)
def test_tc_backward_weight_matches_oracle(mpm, box, cin, cout):
    """The tensor-core weight and bias gradients against the FP64 oracle on the same BF16 values: the
    products are exact in FP32, so only the FP32 accumulation order differs. The last three boxes hold more
    tiles than there are SMs, so each CTA adds several tiles into its tensor-memory accumulators."""
    cd = 4 if cout <= 4 else (16 if cout <= 16 else 32)
    x = torch.from_numpy(RNG.normal(size=box + (cin,)).astype(np.float32)).to(torch.bfloat16).cuda()
    dy = torch.from_numpy(RNG.normal(size=box + (cout,)).astype(np.float32)).to(torch.bfloat16).cuda()
    dyp = torch.zeros(box + (cd,), dtype=torch.bfloat16, device="cuda")
    dyp[..., :cout] = dy
    dw = torch.full((27, cout, cin), 5.0, dtype=torch.float32, device="cuda")  # overwritten
    db = torch.full((cout,), 5.0, dtype=torch.float32, device="cuda")
    mpm.mpm_conv3d_backward_weight_tc(*box, cin, cout, x.data_ptr(), dyp.data_ptr(), dw.data_ptr(), db.data_ptr())
    assert mpm.mpm_net_tc_status(clear=1) == 0
    ref_w, ref_b = no.conv3d_backward_weight(x.float().cpu().numpy(), dy.float().cpu().numpy())
    got_w, got_b = dw.cpu().numpy(), db.cpu().numpy()
    print(f"box {box} {cin}->{cout}: dw rel {rel(got_w, ref_w):.2e}, db rel {rel(got_b, ref_b):.2e}")
    assert rel(got_w, ref_w) <= 1e-5
    assert rel(got_b, ref_b) <= 1e-5
    # every tap and channel pair, not only the norm: the largest error per entry against the entry scale
    assert np.max(np.abs(got_w - ref_w)) <= 1e-5 * np.max(np.abs(ref_w)) * 8


def test_tc_backward_weight_rejects_bad_shapes(mpm):
    x = torch.zeros(64, dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros(27 * 32 * 32, dtype=torch.float32, device="cuda")
    for cin, cout in ((8, 32), (32, 0), (32, 33)):
        with pytest.raises(mpm.MpmError):
            mpm.mpm_conv3d_backward_weight_tc(1, 1, 1, cin, cout, x.data_ptr(), x.data_ptr(), dw.data_ptr(),
                                              dw.data_ptr())
