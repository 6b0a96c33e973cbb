"""The learned warm start's tensor-core U-Net against the FP64 oracle.

- every convolution kind (plain, concatenated with an upsampled source,
  fp32 / bf16 output, bias and ReLU, backward-data as a convolution with the
  tap-flipped transposed weights) and its weight gradient, on the same
  bf16-rounded operands as the oracle: FP32 accumulation order only;
- the whole network's loss and prediction within 1e-2 relative, and the
  gradient of every parameter tensor within 3e-2 relative (norm-wise): bf16
  activations and bf16 gradient operands put about twenty roundings of up to
  2^-9 on the path from the loss to the deepest layers (measured: 0.1% at
  the head, up to 2.4% at the bottleneck);
- the FP32 debug mode (FP32 activations and weights, CUDA-core
  convolutions, the same element-wise kernels): loss, prediction and the
  gradient of every parameter tensor within 1e-5 relative of the FP64
  oracle, on parameters whose every ReLU decision has a margin of at least
  0.5 (checked in the oracle), so that FP32 rounding cannot flip a mask;
- a few Adam steps lower the loss;
- the TMA-fed kernels on halo-layout tensors equal the cp.async kernels:
  forward bitwise (periodic copies included), weight gradient to FP32
  accumulation order;
- the bulk-copy kernels on planar tensors (the network's own path) equal the
  cp.async kernels to FP32 accumulation order (input channels in stages of
  16, taps inside each); a bf16 output touches exactly the interior and the
  periodic copies.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L
    from paper_1007_1388_gb300 import unet

    L.use_torch_allocator()
    return torch, unet


def _bf16(torch, a):
    """numpy float array -> (CUDA bf16 tensor, float64 numpy of the rounded values)."""
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


def _grid_np(a, nb, lz, ly, lx, c):
    return a.reshape(nb, 1 << lz, 1 << ly, 1 << lx, c)


CASES = [  # (c0, up0, c1, cout, grid (nb, lz, ly, lx), relu, bias, out_f32)
    (16, 0, 0, 16, (2, 3, 4, 4), True, True, False),
    (16, 0, 0, 32, (1, 4, 3, 4), False, True, True),
    (32, 0, 0, 64, (2, 3, 3, 3), True, True, True),
    (64, 1, 32, 32, (2, 3, 4, 3), True, True, True),
    (32, 1, 16, 16, (1, 4, 4, 4), False, False, True),
    (16, 0, 0, 48, (2, 3, 4, 4), False, False, True),
    (32, 0, 0, 96, (1, 3, 4, 4), False, False, True),
    (96, 0, 0, 32, (1, 3, 3, 4), True, True, False),
]


def _ref_input(src0, up0, src1, nb):
    parts = []
    for b in range(nb):
        x = src0[b]
        if up0:
            x = U.up(x)
        if src1 is not None:
            x = np.concatenate([x, src1[b]], axis=-1)
        parts.append(x)
    return parts


@pytest.mark.parametrize("case", CASES)
def test_conv3_forward_matches_oracle(env, case):
    torch, unet = env
    c0, up0, c1, cout, grid, relu, bias, out_f32 = case
    nb, lz, ly, lx = grid
    rng = np.random.default_rng(hash(case) % 2**32)
    V = nb << (lz + ly + lx)
    h = 1 if up0 else 0
    s0, s0r = _bf16(torch, rng.normal(size=(V >> (3 * h)) * c0))
    s1, s1r = (_bf16(torch, rng.normal(size=V * c1)) if c1 else (None, None))
    w, wr = _bf16(torch, rng.normal(0, 0.1, size=cout * 27 * (c0 + c1)))
    b = torch.from_numpy(rng.normal(size=cout).astype(np.float32)).cuda() if bias else None
    out = torch.empty(V * cout, dtype=torch.float32 if out_f32 else torch.bfloat16, device="cuda")
    unet.conv3(s0, c0, w, out, cout, grid, up0=bool(up0), src1=s1, c1=c1, bias=b, relu=relu)
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().reshape(nb, -1, cout)
    x0 = _grid_np(s0r, nb, lz - h, ly - h, lx - h, c0)
    x1 = _grid_np(s1r, nb, lz, ly, lx, c1) if c1 else None
    W = wr.reshape(cout, 27, c0 + c1)
    bb = b.cpu().numpy().astype(np.float64) if bias else np.zeros(cout)
    for k, x in enumerate(_ref_input(x0, up0, x1, nb)):
        ref = U.conv(x, W, bb)
        if relu:
            ref = U.relu(ref)
        ref = ref.reshape(-1, cout)
        # scale of the terms summed: sum |x||w| per output
        mag = np.abs(U.conv(np.abs(x), np.abs(W), np.abs(bb))).reshape(-1, cout)
        tol = (2e-6 * mag + 1e-6) if out_f32 else (np.abs(ref) * 2.0**-8 + 2e-6 * mag + 1e-6)
        err = np.abs(got[k] - ref)
        assert np.all(err <= tol), (case, float((err / (mag + 1e-9)).max()))


@pytest.mark.parametrize("case", [c for c in CASES if c[3] <= 64][:5])
def test_conv3_weight_gradient_matches_oracle(env, case):
    torch, unet = env
    c0, up0, c1, cout, grid, _, _, _ = case
    nb, lz, ly, lx = grid
    rng = np.random.default_rng(7 + hash(case) % 2**31)
    V = nb << (lz + ly + lx)
    h = 1 if up0 else 0
    s0, s0r = _bf16(torch, rng.normal(size=(V >> (3 * h)) * c0))
    s1, s1r = (_bf16(torch, rng.normal(size=V * c1)) if c1 else (None, None))
    dy, dyr = _bf16(torch, rng.normal(size=V * cout))
    dw = torch.empty(cout * 27 * (c0 + c1), dtype=torch.float32, device="cuda")
    unet.conv3_wgrad(s0, c0, dy, cout, dw, grid, up0=bool(up0), src1=s1, c1=c1)
    got = dw.cpu().numpy().reshape(cout, 27, c0 + c1)
    x0 = _grid_np(s0r, nb, lz - h, ly - h, lx - h, c0)
    x1 = _grid_np(s1r, nb, lz, ly, lx, c1) if c1 else None
    g = dyr.reshape(nb, 1 << lz, 1 << ly, 1 << lx, cout)
    ref = np.zeros_like(got, dtype=np.float64)
    mag = np.zeros_like(ref)
    W0 = np.zeros((cout, 27, c0 + c1))
    for k, x in enumerate(_ref_input(x0, up0, x1, nb)):
        ref += U.conv_backward(x, W0, g[k])[1]
        mag += U.conv_backward(np.abs(x), W0, np.abs(g[k]))[1]
    err = np.abs(got - ref)
    assert np.all(err <= 2e-6 * mag + 1e-6), float((err / (mag + 1e-9)).max())


def test_backward_data_is_the_flipped_convolution(env):
    """The network's backward-data step: conv with wb[ci][t][co] = W[co][26-t][ci]
    equals the oracle's input gradient."""
    torch, unet = env
    rng = np.random.default_rng(11)
    nb, lz, ly, lx, cin, cout = 2, 3, 4, 3, 32, 16
    V = nb << (lz + ly + lx)
    W = rng.normal(0, 0.1, size=(cout, 27, cin))
    dy, dyr = _bf16(torch, rng.normal(size=V * cout))
    wb = np.transpose(W[:, ::-1, :], (2, 1, 0)).copy()  # [cin][27][cout], taps flipped
    wbt, wbr = _bf16(torch, wb)
    out = torch.empty(V * cin, dtype=torch.float32, device="cuda")
    unet.conv3(dy, cout, wbt, out, cin, (nb, lz, ly, lx))
    got = out.cpu().numpy().reshape(nb, -1, cin)
    Wr = np.transpose(wbr.reshape(cin, 27, cout)[:, ::-1, :], (2, 1, 0))
    g = dyr.reshape(nb, 1 << lz, 1 << ly, 1 << lx, cout)
    x0 = np.zeros((1 << lz, 1 << ly, 1 << lx, cin))
    for k in range(nb):
        ref = U.conv_backward(x0, Wr, g[k])[0].reshape(-1, cin)
        mag = U.conv_backward(x0, np.abs(Wr), np.abs(g[k]))[0].reshape(-1, cin)
        assert np.all(np.abs(got[k] - ref) <= 2e-6 * mag + 1e-6)


def _oracle_params(flat):
    p, o = {}, 0
    for name, ci, co in U.CONVS:
        p[name] = flat[o:o + co * 27 * ci].reshape(co, 27, ci).astype(np.float64)
        o += co * 27 * ci
        p["b" + name[1:]] = flat[o:o + co].astype(np.float64)
        o += co
    p["Wh"] = flat[o:o + 64].reshape(4, 16).astype(np.float64)
    o += 64
    p["bh"] = flat[o:o + 4].astype(np.float64)
    o += 4
    assert o == flat.size
    return p


def _oracle_flat(g):
    parts = []
    for name, _, _ in U.CONVS:
        parts += [g[name].reshape(-1), g["b" + name[1:]].reshape(-1)]
    parts += [g["Wh"].reshape(-1), g["bh"].reshape(-1)]
    return np.concatenate(parts)


def _sample_inputs(rng, n, nb):
    from paper_1007_1388_gb300 import workloads as W

    solid = np.stack([W.sphere_packing(rng, (n, n, n), 0.8, 2, 3) for _ in range(nb)])
    # the network's input channels are bf16: take forces that bf16 represents
    force = (np.round(rng.uniform(0.2, 1.0, nb) * 128) / 128).astype(np.float32)
    target = rng.normal(0, 0.5, size=(nb, n, n, n, 4)).astype(np.float32)
    return solid, force, target


def test_network_loss_and_gradients_match_oracle(env):
    torch, unet = env
    n, nb = 16, 2
    rng = np.random.default_rng(21)
    net = unet.UNet(n, nb, seed=5)
    flat = net.get_params()
    # nonzero biases so that every bias path is exercised
    p = _oracle_params(flat.copy())
    for k in p:
        if k.startswith("b"):
            p[k][:] = rng.normal(0, 0.05, p[k].shape)
    flat = _oracle_flat(p).astype(np.float32)
    net.set_params(flat)
    p = _oracle_params(flat)
    solid, force, target = _sample_inputs(rng, n, nb)
    loss, g = net.loss_grad(torch.from_numpy(solid.reshape(-1)).cuda(), force,
                            torch.from_numpy(target.reshape(-1)).cuda(), grads=True)
    ref_loss, ref_g = 0.0, None
    for b in range(nb):
        x = np.zeros((n, n, n, 2))
        x[..., 0] = solid[b] != 0
        x[..., 1] = np.float32(np.asarray(force[b], np.float32).astype(np.float32))
        y, a = U.forward(p, x)
        ref_loss += U.loss(y, target[b]) / nb
        gb = _oracle_flat(U.backward(p, a, y, target[b])) / nb
        ref_g = gb if ref_g is None else ref_g + gb
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    rp = _oracle_params(ref_g)
    gp = _oracle_params(g.astype(np.float64))
    rels = {k: float(np.linalg.norm(gp[k] - rp[k]) / max(np.linalg.norm(rp[k]), 1e-30)) for k in rp}
    print("gradient relative errors", rels)
    bad = {k: v for k, v in rels.items() if not v <= 3e-2}
    assert not bad, bad
    net.destroy()


def _margin_params(rng):
    """Parameters whose ReLU decisions all have a wide margin: every channel's
    bias is +1 (three of four channels) or -1, the weights are small, so each
    pre-activation stays near its bias while the convolutions still carry the
    inputs' spatial structure."""
    p = {}
    for name, ci, co in U.CONVS:
        p[name] = rng.normal(0, 0.12 / np.sqrt(27 * ci), (co, 27, ci))
        p["b" + name[1:]] = np.where(np.arange(co) % 4 == 3, -1.0, 1.0) + rng.normal(0, 0.05, co)
    p["Wh"] = rng.normal(0, 0.25, (4, 16))
    p["bh"] = rng.normal(0, 0.05, 4)
    return p


def _relu_margin(p, a):
    """Smallest |pre-activation| over every ReLU of the oracle's forward pass."""
    worst = np.inf
    for na, nb, key in (("W1a", "W1b", "e1"), ("W2a", "W2b", "e2"), ("W3a", "W3b", "e3"),
                        ("W4a", "W4b", "d2"), ("W5a", "W5b", "d1")):
        for name, inp in ((na, a[key + "_in"]), (nb, a[key + "_h"])):
            worst = min(worst, float(np.min(np.abs(U.conv(inp, p[name], p["b" + name[1:]])))))
    return worst


def test_f32_debug_mode_gradients_match_oracle_to_1e5(env):
    torch, unet = env
    n, nb = 16, 2
    rng = np.random.default_rng(3)
    flat = _oracle_flat(_margin_params(rng)).astype(np.float32)
    p = _oracle_params(flat)
    solid, force, target = _sample_inputs(rng, n, nb)
    net = unet.UNet(n, nb, seed=1, precision=unet.F32)
    net.set_params(flat)
    sd = torch.from_numpy(solid.reshape(-1)).cuda()
    out = torch.empty(nb * n**3 * 4, dtype=torch.float32, device="cuda")
    net.predict(sd, force, out)
    got = out.cpu().numpy().reshape(nb, -1, 4)
    loss, g = net.loss_grad(sd, force, torch.from_numpy(target.reshape(-1)).cuda(), grads=True)
    ref_loss, ref_g = 0.0, None
    for b in range(nb):
        x = np.zeros((n, n, n, 2))
        x[..., 0] = solid[b] != 0
        x[..., 1] = np.float64(force[b])
        y, a = U.forward(p, x)
        assert _relu_margin(p, a) > 0.5
        assert np.linalg.norm(got[b] - y.reshape(-1, 4)) <= 1e-6 * np.linalg.norm(y)
        ref_loss += U.loss(y, target[b]) / nb
        gb = _oracle_flat(U.backward(p, a, y, target[b])) / nb
        ref_g = gb if ref_g is None else ref_g + gb
    assert abs(loss - ref_loss) <= 1e-6 * ref_loss
    rp = _oracle_params(ref_g)
    gp = _oracle_params(g.astype(np.float64))
    rels = {k: float(np.linalg.norm(gp[k] - rp[k]) / max(np.linalg.norm(rp[k]), 1e-30)) for k in rp}
    print("FP32 gradient relative errors", rels)
    bad = {k: v for k, v in rels.items() if not v <= 1e-5}
    assert not bad, bad
    net.destroy()


def test_prediction_matches_oracle_and_training_lowers_loss(env):
    torch, unet = env
    n, nb = 16, 2
    rng = np.random.default_rng(33)
    net = unet.UNet(n, nb, seed=9)
    p = _oracle_params(net.get_params())
    solid, force, target = _sample_inputs(rng, n, nb)
    sd = torch.from_numpy(solid.reshape(-1)).cuda()
    out = torch.empty(nb * n**3 * 4, dtype=torch.float32, device="cuda")
    net.predict(sd, force, out)
    got = out.cpu().numpy().reshape(nb, -1, 4)
    for b in range(nb):
        x = np.zeros((n, n, n, 2))
        x[..., 0] = solid[b] != 0
        x[..., 1] = force[b]
        y, _ = U.forward(p, x)
        y = y.reshape(-1, 4)
        assert np.linalg.norm(got[b] - y) <= 1e-2 * np.linalg.norm(y)
    tg = torch.from_numpy(target.reshape(-1)).cuda()
    l0 = net.train_step(sd, force, tg, 1e-3)
    for _ in range(30):
        l1 = net.train_step(sd, force, tg, 1e-3)
    assert l1 < 0.9 * l0, (l0, l1)
    net.destroy()


# ------------------------------------------------------------- TMA-fed (halo layout)
def _to_halo(torch, t, nb, lz, ly, lx, c):
    """(nb*nz*ny*nx*c) -> halo layout [nb][nz+2][ny][nx+2][c] with periodic x/z copies."""
    a = t.view(nb, 1 << lz, 1 << ly, 1 << lx, c)
    a = torch.cat([a[:, :, :, -1:], a, a[:, :, :, :1]], dim=3)
    a = torch.cat([a[:, -1:], a, a[:, :1]], dim=1)
    return a.contiguous().view(-1)


def _from_halo(torch, t, nb, lz, ly, lx, c):
    a = t.view(nb, (1 << lz) + 2, 1 << ly, (1 << lx) + 2, c)
    return a[:, 1:-1, :, 1:-1].contiguous().view(-1)


@pytest.mark.parametrize("case", [c for c in CASES if not c[1]])
def test_tma_conv3_equals_cpasync_conv3(env, case):
    torch, unet = env
    c0, _, c1, cout, grid, relu, bias, out_f32 = case
    nb, lz, ly, lx = grid
    rng = np.random.default_rng(17 + hash(case) % 2**31)
    V = nb << (lz + ly + lx)
    s0, _ = _bf16(torch, rng.normal(size=V * c0))
    s1, _ = (_bf16(torch, rng.normal(size=V * c1)) if c1 else (None, None))
    w, _ = _bf16(torch, rng.normal(0, 0.1, size=cout * 27 * (c0 + c1)))
    b = torch.from_numpy(rng.normal(size=cout).astype(np.float32)).cuda() if bias else None
    dt = torch.float32 if out_f32 else torch.bfloat16
    ref = torch.empty(V * cout, dtype=dt, device="cuda")
    unet.conv3(s0, c0, w, ref, cout, grid, src1=s1, c1=c1, bias=b, relu=relu)
    h0 = _to_halo(torch, s0, nb, lz, ly, lx, c0)
    h1 = _to_halo(torch, s1, nb, lz, ly, lx, c1) if c1 else None
    if out_f32:
        got = torch.empty(V * cout, dtype=dt, device="cuda")
        unet.conv3_halo(h0, c0, w, got, cout, grid, src1=h1, c1=c1, bias=b, relu=relu)
        assert torch.equal(got, ref)
    else:
        n_h = nb * ((1 << lz) + 2) * (1 << ly) * ((1 << lx) + 2) * cout
        got = torch.full((n_h,), float("nan"), dtype=dt, device="cuda")
        unet.conv3_halo(h0, c0, w, got, cout, grid, src1=h1, c1=c1, bias=b, relu=relu)
        torch.cuda.synchronize()
        assert torch.equal(got, _to_halo(torch, ref, nb, lz, ly, lx, cout))  # interior and periodic copies


@pytest.mark.parametrize("case", [c for c in CASES if not c[1] and c[3] <= 64])
def test_tma_wgrad_equals_cpasync_wgrad(env, case):
    torch, unet = env
    c0, _, c1, cout, grid, _, _, _ = case
    nb, lz, ly, lx = grid
    rng = np.random.default_rng(23 + hash(case) % 2**31)
    V = nb << (lz + ly + lx)
    s0, _ = _bf16(torch, rng.normal(size=V * c0))
    s1, _ = (_bf16(torch, rng.normal(size=V * c1)) if c1 else (None, None))
    dy, _ = _bf16(torch, rng.normal(size=V * cout))
    ref = torch.empty(cout * 27 * (c0 + c1), dtype=torch.float32, device="cuda")
    unet.conv3_wgrad(s0, c0, dy, cout, ref, grid, src1=s1, c1=c1)
    got = torch.empty_like(ref)
    unet.conv3_halo_wgrad(_to_halo(torch, s0, nb, lz, ly, lx, c0), c0, _to_halo(torch, dy, nb, lz, ly, lx, cout),
                          cout, got, grid, src1=_to_halo(torch, s1, nb, lz, ly, lx, c1) if c1 else None, c1=c1)
    # same products, the splits may differ: FP32 accumulation order only
    mag = float(ref.abs().max())
    assert float((got - ref).abs().max()) <= 1e-5 * mag + 1e-6


# ------------------------------------------------------------- bulk copies (planar layout)
def _to_planar(torch, unet, t, grid, c, copies=True):
    """(nb*nz*ny*nx*c) channels-last -> planar [c/8][P][8]: periodic x/z copies
    (or zeros without `copies`), zero wall rows and guards."""
    nb, lz, ly, lx = grid
    a = t.view(nb, 1 << lz, 1 << ly, 1 << lx, c)
    if copies:
        a = torch.cat([a[:, :, :, -1:], a, a[:, :, :, :1]], dim=3)
        a = torch.cat([a[:, -1:], a, a[:, :1]], dim=1)
    else:
        zx = torch.zeros_like(a[:, :, :, :1])
        a = torch.cat([zx, a, zx], dim=3)
        zz = torch.zeros_like(a[:, :1])
        a = torch.cat([zz, a, zz], dim=1)
    z = torch.zeros_like(a[:, :, :1])
    a = torch.cat([z, a, z], dim=2).reshape(-1, c // 8, 8).permute(1, 0, 2)
    out = torch.zeros(c // 8, unet.planar_positions(grid), 8, dtype=t.dtype, device=t.device)
    g0 = 1024 + ((1 << ly) + 2) * ((1 << lx) + 2) + (1 << lx) + 2
    out[:, g0:g0 + a.shape[1]] = a
    return out.reshape(-1)


def _pack(torch, w, cout, cin):
    """bf16 [cout][27][cin] -> [cin/16][9][2][3][cout][8] (tap t = 3 p + d)."""
    return w.view(cout, 9, 3, cin // 16, 2, 8).permute(3, 1, 4, 2, 0, 5).contiguous().view(-1)


@pytest.mark.parametrize("case", [c for c in CASES if not c[1]])
def test_planar_conv3_matches_cpasync_conv3(env, case):
    torch, unet = env
    c0, _, c1, cout, grid, relu, bias, out_f32 = case
    nb, lz, ly, lx = grid
    rng = np.random.default_rng(29 + hash(case) % 2**31)
    V = nb << (lz + ly + lx)
    s0, _ = _bf16(torch, rng.normal(size=V * c0))
    s1, _ = (_bf16(torch, rng.normal(size=V * c1)) if c1 else (None, None))
    w, _ = _bf16(torch, rng.normal(0, 0.1, size=cout * 27 * (c0 + c1)))
    b = torch.from_numpy(rng.normal(size=cout).astype(np.float32)).cuda() if bias else None
    dt = torch.float32 if out_f32 else torch.bfloat16
    ref = torch.empty(V * cout, dtype=dt, device="cuda")
    unet.conv3(s0, c0, w, ref, cout, grid, src1=s1, c1=c1, bias=b, relu=relu)
    p0 = _to_planar(torch, unet, s0, grid, c0)
    p1 = _to_planar(torch, unet, s1, grid, c1) if c1 else None
    wpk = _pack(torch, w, cout, c0 + c1)
    if out_f32:
        got = torch.empty(V * cout, dtype=dt, device="cuda")
        unet.conv3_planar(p0, c0, wpk, got, cout, grid, src1=p1, c1=c1, bias=b, relu=relu)
        want = ref
    else:
        got = torch.full((cout * unet.planar_positions(grid),), float("nan"), dtype=dt, device="cuda")
        unet.conv3_planar(p0, c0, wpk, got, cout, grid, src1=p1, c1=c1, bias=b, relu=relu)
        torch.cuda.synchronize()
        # untouched positions (wall rows, guards) stay NaN: count them as zero
        got = torch.nan_to_num(got, nan=0.0)
        want = _to_planar(torch, unet, ref, grid, cout)
    g, r = got.float(), want.float()
    # FP32 order only; a bf16 output may round the other way (one bf16 step)
    tol = (1e-5 if out_f32 else 2.0**-7) * float(r.abs().max())
    assert float((g - r).abs().max()) <= tol
    assert torch.equal(torch.isnan(got), torch.zeros_like(torch.isnan(got)))


@pytest.mark.parametrize("case", [c for c in CASES if not c[1] and c[3] <= 128])
def test_planar_wgrad_matches_cpasync_wgrad(env, case):
    torch, unet = env
    c0, _, c1, cout, grid, _, _, _ = case
    nb, lz, ly, lx = grid
    rng = np.random.default_rng(31 + hash(case) % 2**31)
    V = nb << (lz + ly + lx)
    s0, _ = _bf16(torch, rng.normal(size=V * c0))
    s1, _ = (_bf16(torch, rng.normal(size=V * c1)) if c1 else (None, None))
    dy, _ = _bf16(torch, rng.normal(size=V * cout))
    ref = torch.empty(cout * 27 * (c0 + c1), dtype=torch.float32, device="cuda")
    unet.conv3_wgrad(s0, c0, dy, cout, ref, grid, src1=s1, c1=c1)
    got = torch.empty_like(ref)
    dyz = _to_planar(torch, unet, dy, grid, cout, copies=False)
    unet.conv3_planar_wgrad(_to_planar(torch, unet, s0, grid, c0), c0, dyz, cout, got, grid,
                            src1=_to_planar(torch, unet, s1, grid, c1) if c1 else None, c1=c1)
    mag = float(ref.abs().max())
    assert float((got - ref).abs().max()) <= 1e-5 * mag + 1e-6
