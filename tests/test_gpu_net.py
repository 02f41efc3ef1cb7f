"""GPU parity of the surrogate network kernels (include/mpm_net.h) with the FP64 network oracle.

FP32 reference mode: forward, input gradient, weight gradient, a whole network's gradient, loss and Adam
at 1e-5 relative. BF16 tensor-core mode: the same quantities at 1e-2 relative, both sides fed the same
BF16-rounded inputs (the oracle widens them to FP64), on boxes that are not multiples of the 4 x 4 x 8
tile and on the layer shapes of the surrogate (4 -> 32 -> 32 -> 32 -> 3)."""
import numpy as np
import pytest
import torch

from oracle import net_oracle as no

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(77)


@pytest.fixture(scope="module")
def mpm():
    from paper_2302_04659_gb300 import _native, build
    build.build()
    return _native


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.to(dtype).cuda().contiguous()


def as_oracle(t):
    """The exact values the GPU sees (BF16 rounding included), widened to FP64."""
    return t.float().cpu().numpy().astype(np.float64)


SHAPES = [((5, 6, 9), 4, 32), ((4, 4, 8), 32, 32), ((7, 9, 11), 32, 3), ((1, 1, 1), 32, 32), ((3, 5, 17), 3, 32)]


@pytest.mark.parametrize("box,cin,cout", SHAPES)
@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_conv_forward(mpm, box, cin, cout, prec):
    dt = torch.float32 if prec == "f32" else torch.bfloat16
    code = mpm.MPM_NET_F32 if prec == "f32" else mpm.MPM_NET_BF16
    x = dev(RNG.normal(size=box + (cin,)), dt)
    w = dev(0.2 * RNG.normal(size=(27, cout, cin)), dt)
    b = dev(RNG.normal(size=cout), torch.float32)
    for relu in (0, 1):
        y = torch.zeros(box + (cout,), dtype=torch.float32 if prec == "f32" else dt, device="cuda")
        mpm.mpm_conv3d_forward(code, *box, cin, cout, x.data_ptr(), w.data_ptr(), b.data_ptr(), relu, 0,
                               y.data_ptr())
        torch.cuda.synchronize()
        ref = no.conv3d_forward(as_oracle(x), as_oracle(w), as_oracle(b))
        if relu:
            ref = no.relu(ref)
        tol = 1e-5 if prec == "f32" else 1e-2
        assert rel(as_oracle(y), ref) <= tol
    if prec == "bf16":  # FP32 output of the BF16 kernel: only the accumulation order differs
        y = torch.zeros(box + (cout,), dtype=torch.float32, device="cuda")
        mpm.mpm_conv3d_forward(code, *box, cin, cout, x.data_ptr(), w.data_ptr(), b.data_ptr(), 0, 1, y.data_ptr())
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), no.conv3d_forward(as_oracle(x), as_oracle(w), as_oracle(b))) <= 1e-5


@pytest.mark.parametrize("box,cin,cout", SHAPES)
@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_conv_backward(mpm, box, cin, cout, prec):
    dt = torch.float32 if prec == "f32" else torch.bfloat16
    code = mpm.MPM_NET_F32 if prec == "f32" else mpm.MPM_NET_BF16
    tol = 1e-5 if prec == "f32" else 1e-2
    x = dev(np.maximum(RNG.normal(size=box + (cin,)), 0.0), dt)  # a ReLU output: also the mask
    w = dev(0.2 * RNG.normal(size=(27, cout, cin)), dt)
    dy = dev(RNG.normal(size=box + (cout,)), dt)
    dx = torch.zeros(box + (cin,), dtype=dt, device="cuda")
    mpm.mpm_conv3d_backward_data(code, *box, cin, cout, dy.data_ptr(), w.data_ptr(), 0, dx.data_ptr())
    dxm = torch.zeros_like(dx)
    mpm.mpm_conv3d_backward_data(code, *box, cin, cout, dy.data_ptr(), w.data_ptr(), x.data_ptr(), dxm.data_ptr())
    dw = torch.zeros((27, cout, cin), dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    mpm.mpm_conv3d_backward_weight(code, *box, cin, cout, x.data_ptr(), dy.data_ptr(), dw.data_ptr(), db.data_ptr())
    torch.cuda.synchronize()
    ref_dx = no.conv3d_backward_data(as_oracle(dy), as_oracle(w))
    assert rel(as_oracle(dx), ref_dx) <= tol
    assert rel(as_oracle(dxm), no.relu_backward(ref_dx, as_oracle(x))) <= tol
    ref_dw, ref_db = no.conv3d_backward_weight(as_oracle(x), as_oracle(dy))
    # weight gradients accumulate in FP32 from exact BF16 products: FP32-level agreement in both modes
    assert rel(dw.cpu().numpy(), ref_dw) <= 1e-5
    assert rel(db.cpu().numpy(), ref_db) <= 1e-5


def net_params(rng):
    chans = [4, 32, 32, 32, 3]
    return [(0.15 * rng.normal(size=(27, chans[i + 1], chans[i])), 0.05 * rng.normal(size=chans[i + 1]))
            for i in range(4)]


def gpu_network_gradient(mpm, params, x, target, mask, prec):
    """Forward, loss and backward through the C-ABI kernels. Returns (loss, [(dw, db)], output)."""
    dt = torch.float32 if prec == "f32" else torch.bfloat16
    code = mpm.MPM_NET_F32 if prec == "f32" else mpm.MPM_NET_BF16
    box = x.shape[:3]
    chans = [4, 32, 32, 32, 3]
    W = [dev(w, dt) for w, _ in params]
    B = [dev(b, torch.float32) for _, b in params]
    acts = [dev(x, dt)]
    for i in range(4):
        last = i == 3
        y = torch.zeros(box + (chans[i + 1],), dtype=torch.float32 if last else dt, device="cuda")
        mpm.mpm_conv3d_forward(code, *box, chans[i], chans[i + 1], acts[-1].data_ptr(), W[i].data_ptr(),
                               B[i].data_ptr(), 0 if last else 1, 1 if last else 0, y.data_ptr())
        acts.append(y)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    msk = torch.from_numpy(mask.astype(np.uint8)).cuda()
    loss = torch.zeros(2, dtype=torch.float32, device="cuda")
    g = torch.zeros(box + (3,), dtype=dt, device="cuda")
    nvox = int(np.prod(box))
    mpm.mpm_mse_loss(code, nvox, 3, acts[-1].data_ptr(), 1, tgt.data_ptr(), msk.data_ptr(), loss.data_ptr(),
                     g.data_ptr())
    grads = [None] * 4
    for i in range(3, -1, -1):
        dw = torch.zeros((27, chans[i + 1], chans[i]), dtype=torch.float32, device="cuda")
        db = torch.zeros(chans[i + 1], dtype=torch.float32, device="cuda")
        mpm.mpm_conv3d_backward_weight(code, *box, chans[i], chans[i + 1], acts[i].data_ptr(), g.data_ptr(),
                                       dw.data_ptr(), db.data_ptr())
        grads[i] = (dw, db)
        if i > 0:
            gx = torch.zeros(box + (chans[i],), dtype=dt, device="cuda")
            mpm.mpm_conv3d_backward_data(code, *box, chans[i], chans[i + 1], g.data_ptr(), W[i].data_ptr(),
                                         acts[i].data_ptr(), gx.data_ptr())
            g = gx
    torch.cuda.synchronize()
    return (float(loss[0]), [(a.cpu().numpy(), b.cpu().numpy()) for a, b in grads],
            acts[-1].cpu().numpy(), [as_oracle(w) for w in W], acts)


def bf16(a):
    """Round to BF16 (nearest even) and widen back: the precision of the GPU's stored tensors."""
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def reference_network_gradient(params, x, target, mask, rounded):
    """The oracle's forward, loss and backward; with ``rounded`` every tensor the BF16 path stores
    (input, weights, hidden activations, activation gradients) is rounded to BF16 between the oracle's
    FP64 operations, mirroring where the GPU rounds (accumulation stays exact here, FP32 there)."""
    r = bf16 if rounded else (lambda a: np.asarray(a, np.float64))
    ps = [(r(w), np.asarray(b, np.float32).astype(np.float64)) for w, b in params]
    acts = [r(x)]
    for i, (w, b) in enumerate(ps):
        z = no.conv3d_forward(acts[-1], w, b)
        acts.append(r(no.relu(z)) if i < 3 else z)
    L, g = no.mse_loss(acts[-1], target.astype(np.float32), mask)
    g = r(g)
    grads = [None] * 4
    for i in range(3, -1, -1):
        grads[i] = no.conv3d_backward_weight(acts[i], g)
        if i > 0:
            g = r(no.relu_backward(no.conv3d_backward_data(g, ps[i][0]), acts[i]))
    return L, grads, acts[-1]


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_network_gradient_matches_oracle(mpm, prec):
    rng = np.random.default_rng(5)
    params = net_params(rng)
    box = (6, 7, 10)
    x = rng.normal(size=box + (4,))
    target = rng.normal(size=box + (3,))
    mask = rng.random(box) < 0.5
    loss, grads, out, _, _ = gpu_network_gradient(mpm, params, x, target, mask, prec)
    tol = 1e-5 if prec == "f32" else 1e-2
    L, ref, y = reference_network_gradient(params, x, target, mask, rounded=prec == "bf16")
    assert abs(loss - L) <= tol * L
    assert rel(out, y) <= tol
    for i in range(4):
        assert rel(grads[i][0], ref[i][0]) <= tol, (i, rel(grads[i][0], ref[i][0]))
        assert rel(grads[i][1], ref[i][1]) <= tol, (i, rel(grads[i][1], ref[i][1]))
    if prec == "bf16":
        # against the unrounded FP64 network (a sanity bound, not the parity bar): BF16 storage rounds
        # at 2^-9 relative, seven times in sequence on the way to the first layer's weight gradient, and
        # the sums over voxels cancel, so the first layer sits near 7e-2 on this random network
        L64, ref64, y64 = reference_network_gradient(params, x, target, mask, rounded=False)
        assert rel(out, y64) <= 3e-2
        for i in range(4):
            assert rel(grads[i][0], ref64[i][0]) <= 1e-1


def test_adam_matches_oracle(mpm):
    n = 1000
    p = RNG.normal(size=n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    P, M, V = (torch.from_numpy(a.copy()).cuda() for a in (p, m, v))
    Pb = torch.zeros(n, dtype=torch.bfloat16, device="cuda")
    rp, rm, rv = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 4):
        g = RNG.normal(size=n).astype(np.float32)
        G = torch.from_numpy(g).cuda()
        mpm.mpm_adam_step(n, P.data_ptr(), G.data_ptr(), M.data_ptr(), V.data_ptr(), t, 1e-3, 0.9, 0.999, 1e-8,
                          Pb.data_ptr())
        rp, rm, rv = no.adam_step(rp, g.astype(np.float64), rm, rv, t, 1e-3)
    torch.cuda.synchronize()
    assert np.abs(P.cpu().numpy() - rp).max() <= 1e-6
    assert torch.equal(Pb, P.to(torch.bfloat16))


def test_tiled_forward_matches_full_on_the_mask(mpm):
    """The tiled forward (only tiles near the mask computed) gives the full network's output on the mask."""
    from paper_2302_04659_gb300 import surrogate as sur
    rng = np.random.default_rng(21)
    net = sur.Network(seed=3)
    box = (13, 18, 21)
    x = dev(rng.normal(size=box + (4,)), torch.bfloat16)
    mask = np.zeros(box, np.uint8)
    mask[3:7, 9:12, 2:9] = 1  # a blob in one corner region
    mask[11, 17, 20] = 1
    md = torch.from_numpy(mask).cuda()
    full = net.forward(x).clone()
    tiled = net.forward(x, md).clone()
    torch.cuda.synchronize()
    on = md.bool()
    assert torch.equal(full[on], tiled[on])
    nflags = mpm.mpm_conv3d_tile_count(*box)
    assert nflags == 4 * 3 * 3  # ceil(13/4) * ceil(18/8) * ceil(21/8)
    flags = torch.zeros(nflags, dtype=torch.uint8, device="cuda")
    mpm.mpm_conv3d_tile_flags(*box, md.data_ptr(), 0, flags.data_ptr())
    torch.cuda.synchronize()
    assert 0 < int(flags.sum()) < nflags
