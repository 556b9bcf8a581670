"""GPU tests of the learned importance-sampling proposal through the C ABI:
tensor-core MLP gradients and inference against the FP64 oracle (BF16
tolerances), Adam, training, the proposal table, the sampler (bit-exact
against the oracle's sampler on the same integer proposal), and an
end-to-end check that the importance-weighted cross section agrees with
uniform sampling while reducing its standard error per GPU-second."""
import math

import numpy as np
import pytest

from paper_2304_02731_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NP = 9156
SLICES = {"W1": (0, 512), "b1": (512, 576), "W2": (576, 4672), "b2": (4672, 4736),
          "W3": (4736, 8832), "b3": (8832, 8896), "W4": (8896, 9152), "b4": (9152, 9156)}


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_02731_gb300 import build
    build.build()
    from paper_2304_02731_gb300 import qcams
    qcams.lib()
    return qcams


def _params(seed, scale=0.25):
    return np.random.default_rng(seed).normal(0.0, scale, NP).astype(np.float32)


def _features(n, seed):
    """Raw inputs shaped like (E, b, v, j, theta, phi, chi, eta)."""
    rng = np.random.default_rng(seed)
    E, b, v, j = (rng.uniform(0.05, 0.3, n), np.sqrt(rng.uniform(0, 100, n)),
                  rng.integers(0, 11, n), rng.integers(0, 21, n))
    th = np.arccos(rng.uniform(-1, 1, n))
    ph, ch, et = rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 1, n), rng.uniform(0, 2 * np.pi, n)
    return np.stack([E, b, v, j, th, ph, ch, et], axis=1).astype(np.float32)


def _setup(Q, seed, n):
    import torch
    x = _features(n, seed)
    mean, std = x.mean(0), x.std(0)
    mlp = Q.MLP()
    p = _params(seed + 1)
    mlp.set_params(p)
    mlp.set_standardizer(mean, std)
    xs = (x.astype(np.float64) - mean.astype(np.float64)) / std.astype(np.float64)
    return mlp, p, x, xs, torch.tensor(x).cuda()


def test_mlp_gradient_matches_oracle(Q, oracle):
    """Gradient of the softmax cross-entropy per layer against the FP64
    oracle.  The GPU rounds both operands of every matrix product to BF16
    (relative error up to u = 2^-9, standard deviation u / sqrt(3) per
    element), so a product of non-cancelling sums carries a relative error of
    about u sqrt(2/3); the first layer's gradient sits at the end of the
    longest chain of such products (4 forward, 3 backward, the outer product
    with the inputs: 8), about sqrt(8) u sqrt(2/3) = 4.5e-3.  The bound
    2^-7 = 4u per layer leaves a factor ~1.7 over that; the direction must
    agree to cos > 0.9995."""
    import torch
    n = 2000
    mlp, p, x, xs, xd = _setup(Q, 3, n)
    cls = np.random.default_rng(4).integers(0, 6, n).astype(np.uint8)   # 4, 5 carry no target
    loss = float(mlp.compute_grad(xd, torch.tensor(cls).cuda())[0])
    g = mlp.grad.cpu().numpy().astype(np.float64)
    loss_o, g_o = oracle.mlp_loss_grad(p.astype(np.float64), xs, cls.astype(np.int32))
    assert abs(loss - loss_o) <= 0.01 * loss_o
    for name, (a, b) in SLICES.items():
        ga, go = g[a:b], g_o[a:b]
        rel = np.linalg.norm(ga - go) / np.linalg.norm(go)
        cos = ga @ go / (np.linalg.norm(ga) * np.linalg.norm(go))
        print(f"\n{name}: rel {rel:.3e} cos {cos:.6f}")
        assert rel < 2.0 ** -7 and cos > 0.9995, name


def test_mlp_inference_matches_oracle(Q, oracle):
    n = 4096
    mlp, p, x, xs, xd = _setup(Q, 5, n)
    probs = mlp.infer(xd).cpu().numpy()
    z = oracle.mlp_forward(p.astype(np.float64), xs)
    po = np.exp(z - z.max(1, keepdims=True))
    po /= po.sum(1, keepdims=True)
    assert np.max(np.abs(probs - po)) < 0.02
    assert np.mean(probs.argmax(1) == po.argmax(1)) > 0.97
    assert np.allclose(probs.sum(1), 1.0, atol=1e-5)


def test_adam_first_step(Q, oracle):
    """At t = 1 Adam moves each parameter by -lr g/(|g| + eps): where the
    gradient is well above BF16 noise, GPU and oracle steps agree."""
    import torch
    n = 2000
    mlp, p, x, xs, xd = _setup(Q, 7, n)
    cls = np.random.default_rng(8).integers(0, 4, n).astype(np.uint8)
    lr = 1e-3
    mlp.train_step(xd, torch.tensor(cls).cuda(), lr)
    d_gpu = mlp.params.cpu().numpy().astype(np.float64) - p
    _, g_o = oracle.mlp_loss_grad(p.astype(np.float64), xs, cls.astype(np.int32))
    d_o = -lr * g_o / (np.abs(g_o) + 1e-8)
    big = np.abs(g_o) > 3e-3 * np.abs(g_o).max()
    assert big.sum() > 1000
    assert np.mean(np.sign(d_gpu[big]) == np.sign(d_o[big])) > 0.97
    assert np.allclose(np.abs(d_gpu[big]), lr, rtol=2e-2)
    assert mlp.step == 1


def test_training_learns_a_separable_rule(Q):
    """Four classes by the quadrant of (x0, x1): a few hundred Adam steps
    bring the loss far below ln 4 and the accuracy above 90 %."""
    import torch
    rng = np.random.default_rng(9)
    n = 32768
    x = rng.normal(0, 1, (n, 8)).astype(np.float32)
    lab = ((x[:, 0] > 0).astype(int) + 2 * (x[:, 1] > 0).astype(int)).astype(np.uint8)
    xd, ld = torch.tensor(x).cuda(), torch.tensor(lab).cuda()
    mlp = Q.MLP(seed=3)
    mlp.set_standardizer(np.zeros(8), np.ones(8))
    first = None
    for it in range(300):
        idx = torch.randint(0, n, (2048,), device="cuda")
        loss = float(mlp.train_step(xd[idx].contiguous(), ld[idx].contiguous(), 3e-3)[0])
        first = loss if first is None else first
    acc = np.mean(mlp.infer(xd).cpu().numpy().argmax(1) == lab)
    print(f"\nloss {first:.3f} -> {loss:.3f}, accuracy {acc:.4f}")
    assert loss < 0.3 * first and acc > 0.9


def test_device_training_loop(Q):
    """qcams_mlp_train: its minibatch is the rows idx drawn on the device
    (uniform on [0, n), checked by a chi-square test), its gradient equals
    qcams_mlp_grad on the gathered rows, and many steps learn the separable
    rule as well as host-driven steps do."""
    import torch
    rng = np.random.default_rng(19)
    n = 1000
    x = torch.tensor(rng.normal(0, 1, (n, 8)).astype(np.float32)).cuda()
    lab = torch.tensor(rng.integers(0, 6, n).astype(np.uint8)).cuda()
    a, b = Q.MLP(seed=5), Q.MLP(seed=5)
    for m in (a, b):
        m.set_standardizer(np.zeros(8), np.ones(8))
    losses, idx = a.train(x, lab, 1, 200_000, 1e-3, seed=8)
    ih = idx.cpu().numpy()
    assert ih.min() >= 0 and ih.max() < n
    counts = np.bincount(ih, minlength=n)
    chi2 = ((counts - 200.0) ** 2 / 200.0).sum()
    assert chi2 < n + 5 * math.sqrt(2 * n), chi2      # dof = n - 1
    loss_b = float(b.compute_grad(x[idx].contiguous(), lab[idx].contiguous())[0])
    ga, gb = a.grad.cpu().numpy(), b.grad.cpu().numpy()
    assert abs(float(losses[0]) - loss_b) <= 1e-5 * abs(loss_b)
    assert np.allclose(ga, gb, rtol=1e-4, atol=1e-7 * np.abs(gb).max())
    assert a.step == 1
    # learning on device-drawn minibatches
    m = 32768
    xs = rng.normal(0, 1, (m, 8)).astype(np.float32)
    ls = ((xs[:, 0] > 0).astype(int) + 2 * (xs[:, 1] > 0).astype(int)).astype(np.uint8)
    xd, ld = torch.tensor(xs).cuda(), torch.tensor(ls).cuda()
    net = Q.MLP(seed=3)
    net.set_standardizer(np.zeros(8), np.ones(8))
    lo, _ = net.train(xd, ld, 300, 2048, 3e-3, seed=1)
    lo = lo.cpu().numpy()
    acc = np.mean(net.infer(xd).cpu().numpy().argmax(1) == ls)
    print(f"\ndevice loop: loss {lo[0]:.3f} -> {lo[-10:].mean():.3f}, accuracy {acc:.4f}")
    assert lo[-10:].mean() < 0.3 * lo[0] and acc > 0.9 and net.step == 300


def test_proposal_matches_oracle(Q, oracle):
    dims = (8, 4, 4, 4, 2)
    mlp, p, x, xs, xd = _setup(Q, 11, 1024)
    mean, std = mlp.standardizer
    spec = Q.proposal_spec(0.1, 3, 5, dims=dims, b2_max=100.0, eps=1e-3, alpha=0.2)
    q, qfix, cdf = mlp.build_proposal(spec)
    q, qfix, cdf = q.cpu().numpy(), qfix.cpu().numpy(), cdf.cpu().numpy()
    xc = oracle.proposal_grid(dims, 100.0, 0.1, 3, 5, mean, std)
    qo = oracle.proposal(p.astype(np.float64), xc, 1e-3, 0.2)
    N = int(np.prod(dims))
    assert abs(q.sum() - 1.0) < 1e-12 and np.all(q >= 0.2 / N * (1 - 1e-12))
    assert np.max(np.abs(q / qo - 1.0)) < 0.03
    assert np.array_equal(qfix, np.rint(q * 2.0 ** 40).astype(np.int64))
    assert np.array_equal(cdf, np.cumsum(qfix))


def test_sampler_bit_exact_against_oracle(Q, oracle):
    import torch
    dims = (16, 8, 8, 8, 4)
    N = int(np.prod(dims))
    q = np.random.default_rng(12).uniform(0.1, 4.0, N)
    q /= q.sum()
    qfix, cdf = oracle.proposal_cdf(q)
    spec = Q.proposal_spec(0.1, 0, 0, dims=dims, b2_max=100.0)
    n = 100_003
    b, u, w, cell = Q.sample_proposal(spec, torch.tensor(qfix).cuda(), torch.tensor(cdf).cuda(),
                                      n, seed=77, id_offset=5)
    bo, uo, wo, co = oracle.sample_proposal(dims, 100.0, qfix, cdf, n, seed=77, id_offset=5)
    assert np.array_equal(cell.cpu().numpy(), co)
    assert np.array_equal(w.cpu().numpy(), wo)
    assert np.array_equal(u.cpu().numpy().T, uo)
    assert np.allclose(b.cpu().numpy(), bo, rtol=2.3e-16, atol=0)


def test_learned_proposal_is_unbiased_and_gains(Q):
    """Train on LJ(12,6) Ca-H lanes drawn like the mixed study, build the
    proposal at E = 0.10 hartree for the most reactive (v, j), and estimate
    sigma_R = sigma(AC+B) + sigma(BC+A) with it and with uniform sampling:
    the two agree within 3 combined standard errors and the proposal gives
    a smaller standard error per GPU-second."""
    from paper_2304_02731_gb300 import learned as L
    import torch
    spec_sys = W.SYS_H2_CA_LJ12
    x, cls, host = L.generate(spec_sys, 120_000, seed=21)
    mlp = Q.MLP(seed=1)
    losses = L.train(mlp, x, cls, epochs=6, batch=4096, lr=2e-3)
    v, j, frac = L.best_state(host)
    spec = Q.proposal_spec(0.10, v, j)
    n = 40_000
    est_u = L.estimate_uniform(spec_sys, spec, n, seed=31)
    est_q = L.estimate_is(spec_sys, mlp, spec, n, seed=32)
    # second runs: timings without the first-call set-up
    est_u = L.estimate_uniform(spec_sys, spec, n, seed=33)
    est_q = L.estimate_is(spec_sys, mlp, spec, n, seed=34)
    print(f"\nloss {losses[0]:.4f} -> {losses[-1]:.4f}; (v, j) = ({v}, {j}) reactive fraction "
          f"{frac:.3f}\nuniform: sigma_R {est_u.sigma:.4f} +- {est_u.se:.4f} ({est_u.n_reactive} "
          f"reactive, {est_u.seconds:.3f} s)\nlearned: sigma_R {est_q.sigma:.4f} +- {est_q.se:.4f} "
          f"({est_q.n_reactive} reactive, {est_q.seconds:.3f} s)\nFOM ratio "
          f"{est_q.fom / est_u.fom:.2f}, SE ratio {est_u.se / est_q.se:.2f}")
    assert losses[-1] < losses[0]
    assert abs(est_q.sigma - est_u.sigma) <= 3 * np.hypot(est_q.se, est_u.se)
    assert est_q.se < est_u.se
