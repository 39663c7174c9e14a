"""BF16 tensor-core U-Net kernels (learned initial guess) against the FP64
reference, training, and the guessed forward solve.

Tolerances: inputs and weights are bf16 values on both sides, products are
exact and the sums are fp32 on the GPU, so a single convolution (fp32
output) agrees to ~1e-6 relative; we allow 1e-5 of the output scale.  The
full network rounds every activation to bf16 on both sides at the same
points, but a different summation order can flip a rounding, so the
prediction agrees to ~1e-2 of its scale."""
import numpy as np
import pytest

import oracle.unet_oracle as UO
import qpat_synth as S

torch = pytest.importorskip("torch")
Q = pytest.importorskip("paper_1512_02796_gb300")

pytestmark = pytest.mark.gpu


def _need():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda").to(torch.bfloat16)


@pytest.mark.parametrize("n,cin,cout,relu", [(8, 16, 16, True), (8, 32, 48, False), (16, 16, 8, True),
                                             (8, 192, 64, True), (8, 64, 192, False), (16, 48, 16, True)])
def test_conv3d_forward(n, cin, cout, relu):
    _need()
    rng = np.random.default_rng(cin + cout)
    x = UO.to_bf16(rng.standard_normal((n ** 3, cin)))
    w = UO.to_bf16(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    out = torch.empty((n ** 3, cout), dtype=torch.bfloat16, device="cuda")
    o32 = torch.empty((n ** 3, cout), dtype=torch.float32, device="cuda")
    Q.qpat_conv3d_bf16_dev(_bf(x), _bf(w), torch.tensor(b, device="cuda"), cout, relu, n, out, o32)
    torch.cuda.synchronize()
    ref = UO.conv3d(x, w, b.astype(np.float64), n, relu=relu)
    scale = np.abs(ref).max()
    assert np.abs(o32.cpu().numpy() - ref).max() <= 1e-5 * scale
    # the bf16 output is the rounded fp32 value
    np.testing.assert_array_equal(out.float().cpu().numpy(), UO.to_bf16(o32.cpu().numpy()))


@pytest.mark.parametrize("n,cin,cout", [(8, 16, 16), (16, 48, 16), (8, 192, 64), (8, 96, 32)])
def test_conv3d_weight_gradient(n, cin, cout):
    _need()
    rng = np.random.default_rng(7 + cin)
    x = UO.to_bf16(rng.standard_normal((n ** 3, cin)))
    dy = UO.to_bf16(rng.standard_normal((n ** 3, cout)))
    dw = torch.empty((27, cout, cin), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    part = torch.empty(Q.qpat_conv3d_bf16_wgrad_scratch(n, cin, cout), dtype=torch.float32, device="cuda")
    Q.qpat_conv3d_bf16_wgrad_dev(_bf(x), _bf(dy), n, dw, db, part)
    torch.cuda.synchronize()
    rw, rb = UO.conv3d_wgrad(x, dy, n)
    assert np.abs(dw.cpu().numpy() - rw).max() <= 1e-5 * np.abs(rw).max()
    # db sums bf16 values in fp32 over n^3 voxels
    assert np.abs(db.cpu().numpy() - rb).max() <= 1e-4 * np.abs(rb).max()


def test_data_gradient_is_the_flipped_convolution():
    """The backward-data pass convolves with w_t[tap][ci][co] = w[26 - tap][co][ci]."""
    _need()
    rng = np.random.default_rng(11)
    n, cin, cout = 8, 48, 16
    w = UO.to_bf16(rng.standard_normal((27, cout, cin)) / 10)
    dy = UO.to_bf16(rng.standard_normal((n ** 3, cout)))
    wt = np.ascontiguousarray(np.transpose(w[::-1], (0, 2, 1)))
    out = torch.empty((n ** 3, cin), dtype=torch.bfloat16, device="cuda")
    o32 = torch.empty((n ** 3, cin), dtype=torch.float32, device="cuda")
    Q.qpat_conv3d_bf16_dev(_bf(dy), _bf(wt), None, cin, False, n, out, o32)
    torch.cuda.synchronize()
    ref = UO.conv3d_transpose(dy, w, n)
    assert np.abs(o32.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_unet_forward_matches_reference():
    _need()
    n = 32
    net = Q.UNet(n, seed=3)
    try:
        p = net.get_params()
        rng = np.random.default_rng(5)
        x = np.stack([rng.normal(0, 0.3, n ** 3), rng.normal(0, 0.3, n ** 3),
                      np.maximum(rng.normal(0, 1, n ** 3), 0)], axis=1).astype(np.float32)
        y = torch.empty((1, n ** 3), dtype=torch.float32, device="cuda")
        net.predict(torch.tensor(x[None], device="cuda"), y)
        torch.cuda.synchronize()
        ref = UO.unet_forward(p.astype(np.float64), x.astype(np.float64), n)
        assert np.abs(y.cpu().numpy()[0] - ref).max() <= 2e-2 * max(np.abs(ref).max(), 1e-6)
    finally:
        net.close()


def test_training_lowers_loss_and_guess_saves_iterations():
    _need()
    from paper_1512_02796_gb300 import learned as LG
    n = 32
    cfgs = [S.small_config(n, 20.0, 1, 500 + i) for i in range(20)]
    xyz, tets = cfgs[0].mesh()
    mesh = Q.qpat_mesh(xyz, tets)
    net = Q.UNet(n, seed=1)
    try:
        Xs, Ts = [], []
        for cfg in cfgs:
            kap, mu = cfg.coefficients(xyz)
            flux = np.stack([Q.qpat_flux_patch(mesh, p.center, p.normal, p.half_w, p.amp) for p in cfg.patches])
            x, t = LG.sample(mesh, cfg, kap, mu, flux)
            Xs.append(x)
            Ts.append(t)
        X = torch.cat(Xs[:-2])
        T = torch.cat(Ts[:-2])
        losses = LG.train(net, X, T, steps=150, lr=3e-3, batch=4)
        assert np.mean(losses[-10:]) < 0.2 * np.mean(losses[:3])
        # held-out phantom: same accuracy, fewer PCG iterations
        cfg = cfgs[-1]
        kap, mu = cfg.coefficients(xyz)
        flux = np.stack([Q.qpat_flux_patch(mesh, p.center, p.normal, p.half_w, p.amp) for p in cfg.patches])
        dev = torch.device("cuda")
        k, m, f = (torch.tensor(a, device=dev) for a in (kap, mu, flux))
        x, t = LG.sample(mesh, cfg, kap, mu, flux)
        phi0 = LG.guess(net, x)
        prm = Q.qpat_default_params(precision=0)
        phi_a = torch.empty((1, mesh.N), dtype=torch.float64, device=dev)
        phi_b = torch.empty_like(phi_a)
        h = torch.empty_like(phi_a)
        mesh.reset_stats()
        Q.qpat_forward_dev(mesh, k, m, f, phi_a, h, prm)
        it_plain = mesh.stats()["pcg_iters"]
        mesh.reset_stats()
        Q.qpat_forward_guess_dev(mesh, k, m, f, phi0, phi_b, h, prm)
        it_guess = mesh.stats()["pcg_iters"]
        torch.cuda.synchronize()
        rel = float(torch.linalg.norm(phi_b - phi_a) / torch.linalg.norm(phi_a))
        print(f"pcg iterations plain {it_plain} guessed {it_guess}  rel {rel:.2e}  loss {losses[0]:.3e}->{losses[-1]:.3e}")
        assert rel < 1e-10
        assert it_guess < it_plain
    finally:
        net.close()
        mesh.close()


@pytest.mark.parametrize("n,cin,cout", [(8, 16, 16), (16, 192, 64), (8, 64, 192), (16, 48, 32)])
def test_tcgen05_and_mma_sync_engines_agree(n, cin, cout):
    """The tcgen05 (tensor-memory accumulator) and mma.sync convolutions give
    the same FP32 result up to summation order, and no bounded wait of the
    tcgen05 kernel gave up."""
    _need()
    rng = np.random.default_rng(cin * 7 + cout)
    x = UO.to_bf16(rng.standard_normal((n ** 3, cin)))
    w = UO.to_bf16(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = torch.tensor(rng.standard_normal(cout).astype(np.float32), device="cuda")
    res = []
    try:
        for engine in (0, 1):
            Q.qpat_conv3d_set_engine(engine)
            out = torch.empty((n ** 3, cout), dtype=torch.bfloat16, device="cuda")
            o32 = torch.empty((n ** 3, cout), dtype=torch.float32, device="cuda")
            Q.qpat_conv3d_bf16_dev(_bf(x), _bf(w), b, cout, True, n, out, o32)
            torch.cuda.synchronize()
            res.append(o32.cpu().numpy())
    finally:
        Q.qpat_conv3d_set_engine(0)
    scale = np.abs(res[1]).max()
    assert np.abs(res[0] - res[1]).max() <= 1e-5 * scale
    assert Q.qpat_conv3d_tc_timeouts() == 0


def test_whole_network_gradient_matches_oracle():
    """One training step's parameter gradient (qpat_unet_grad_dev: the mean
    squared error of a 32^3 sample, every layer's weights and biases) against
    the oracle's FP64 reverse pass (oracle.unet_oracle.unet_loss_grad, itself
    pinned by central differences).  The GPU rounds weights, activations and
    data gradients to bf16 (8-bit mantissa, ~4e-3 per rounding) through 15
    layers each way, so the bar is 5e-2 on the whole gradient (measured
    1.6e-2), 2.5e-1 per layer (measured up to 1.2e-1, on the 4^3-voxel
    bottleneck layers, whose few voxels average the rounding least) and a
    cosine above 0.995; a missing or wrongly transposed layer gradient is off
    by O(1)."""
    _need()
    n = 32
    rng = np.random.default_rng(12)
    net = Q.UNet(n, seed=5)
    try:
        p = net.get_params().astype(np.float64)
        x3 = rng.standard_normal((n ** 3, 3))
        t = rng.standard_normal(n ** 3)
        xt = torch.tensor(x3[None].astype(np.float32), device="cuda")
        tt = torch.tensor(t[None].astype(np.float32), device="cuda")
        loss_g, g = net.grad(xt, tt)
    finally:
        net.close()
    loss_o, go = UO.unet_loss_grad(p, x3, t, n)
    g = g.astype(np.float64)
    sizes = [27 * co * ci + co for ci, co, _, _ in UO.SPEC]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    per_layer = [float(np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])) for a, b in zip(offs, offs[1:])]
    whole = float(np.linalg.norm(g - go) / np.linalg.norm(go))
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    print(f"loss {loss_g:.6f} vs {loss_o:.6f}; gradient rel {whole:.2e} cos {cos:.6f}; per layer "
          f"{['%.1e' % v for v in per_layer]}")
    assert abs(loss_g - loss_o) <= 2e-2 * loss_o
    assert whole < 5e-2 and cos > 0.995
    assert max(per_layer) < 2.5e-1


def test_log_output_mode():
    """qpat_unet_set_log_output: the prediction is the exponential of the
    network output (the same output as without the mode), and training in
    log space lowers the loss on a field spanning several decades; a
    negative floor is refused."""
    _need()
    n = 32
    net = Q.UNet(n, seed=7)
    try:
        rng = np.random.default_rng(8)
        x = torch.tensor(rng.normal(0, 0.3, (1, n ** 3, 3)).astype(np.float32), device="cuda")
        y0 = torch.empty((1, n ** 3), dtype=torch.float32, device="cuda")
        y1 = torch.empty_like(y0)
        net.predict(x, y0)
        net.set_log_output(1e-6)
        net.predict(x, y1)
        torch.cuda.synchronize()
        np.testing.assert_allclose(y1.cpu().numpy(), np.exp(y0.cpu().numpy()), rtol=1e-5)
        z = np.arange(n ** 3) // (n * n)
        t = torch.tensor(np.exp(-z / 4.0)[None].astype(np.float32), device="cuda")   # 8 decades
        losses = [net.train_step(x, t, 3e-3) for _ in range(60)]
        assert losses[-1] < 0.3 * losses[0]
        with pytest.raises(Q.QpatError):
            net.set_log_output(-1.0)
    finally:
        net.close()
