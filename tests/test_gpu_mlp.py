"""Learned temperature guess: GPU gradients, Adam step and FP16 inference vs the FP64 oracle,
training on Newton samples, and what the trained network gains over the Newton solve without it
(Newton still decides the result)."""

import numpy as np
import pytest

from oracle.mlp import N_PARAMS, adam_step, forward, loss_and_grad, unpack
from oracle.thermo import Nasa7Gas
from tests._gpu import torch_cuda
from workloads import box_mesh, equispaced_tet_nodes, physical_nodes
from workloads.gas import mixture_primitive_state, seeded_nasa7_mixture
from workloads.mlp import glorot_params, temperature_samples

pytestmark = pytest.mark.gpu


def test_mlp_gradient_matches_oracle():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    rng = np.random.default_rng(0)
    theta = glorot_params(1) + rng.normal(scale=0.05, size=N_PARAMS).astype(np.float32)
    n = 1000  # several blocks and a ragged tail
    X = rng.normal(size=(n, 8)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    grad = torch.zeros(N_PARAMS, device="cuda", dtype=torch.float32)
    loss = torch.zeros(1, device="cuda", dtype=torch.float32)
    dg.dg_mlp_loss_grad(torch.tensor(theta, device="cuda"), torch.tensor(X, device="cuda"),
                        torch.tensor(t, device="cuda"), grad, loss)
    L, g = loss_and_grad(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - L) <= 1e-4 * L
    g_gpu = grad.cpu().numpy().astype(np.float64)
    assert np.abs(g_gpu - g).max() <= 1e-3 * np.abs(g).max()
    # each block of parameters separately (small blocks must not hide in the global max)
    for lo, hi in [(0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 4800), (4800, 4801)]:
        assert np.abs(g_gpu[lo:hi] - g[lo:hi]).max() <= 2e-3 * max(np.abs(g[lo:hi]).max(), 1e-6)


def test_adam_step_matches_oracle():
    """The library's Adam kernel against the FP64 oracle step from the same FP32 inputs, at two step
    numbers; the FP32 update carries a few roundings (relative ~1e-7 of the step) plus the rounding
    of the new parameter (2^-24 of it)."""
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    rng = np.random.default_rng(3)
    for t in (1, 7):
        theta = rng.normal(scale=0.3, size=N_PARAMS).astype(np.float32)
        grad = rng.normal(scale=0.05, size=N_PARAMS).astype(np.float32)
        grad[::97] = 0.0                                  # zero gradients, zero moments: no move
        m = (rng.normal(scale=0.01, size=N_PARAMS) * (t > 1)).astype(np.float32)
        v = (rng.uniform(0, 1e-3, size=N_PARAMS) * (t > 1)).astype(np.float32)
        v[::97] = 0.0
        m[::97] = 0.0
        lr = 3e-3
        th_d, g_d, m_d, v_d = (torch.tensor(a, device="cuda") for a in (theta, grad, m, v))
        dg.dg_mlp_adam_step(t, lr, th_d, g_d, m_d, v_d)
        torch.cuda.synchronize()
        th_w, m_w, v_w = adam_step(theta.astype(np.float64), grad.astype(np.float64), m.astype(np.float64),
                                   v.astype(np.float64), t, np.float64(np.float32(lr)))
        step = np.abs(th_w - theta)
        th_g = th_d.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(th_g - th_w) <= 2e-6 * step + 2.0 ** -23 * np.abs(th_w) + 1e-12)
        # FP32 moments: a few roundings of each term's size (the two terms may cancel)
        assert np.all(np.abs(m_d.cpu().numpy() - m_w) <= 3e-7 * (0.9 * np.abs(m) + 0.1 * np.abs(grad)))
        assert np.all(np.abs(v_d.cpu().numpy() - v_w) <= 3e-7 * (0.999 * v + 0.001 * grad.astype(np.float64) ** 2))
        assert np.all(g_d.cpu().numpy() == 0.0)        # the batch gradient is cleared for the next batch
        assert np.all(th_g[::97] == theta[::97])


def _fp16_guess_error_model(theta, X, u=2.0 ** -11, eps_t=2.0 ** -9):
    """Error of the library's inference against the FP64 forward pass, per sample, in units of the
    normalised output y.  Sources: features and W1, W2 rounded to FP16 (relative u each), products
    accumulated in FP32 (2^-23 of the absolute sum, generous), pre-activations rounded to FP16 (u),
    the hardware tanh on FP16 pairs with absolute error at most eps_t, the last layer in FP32.

    Returns (worst, rss):
      worst - a bound that holds however the errors align (tanh propagated through its largest slope
              1 - tanh^2 on |z| - dz, so it is not a linearisation);
      rss   - the root sum of squares of the first-order contributions when every rounding and tanh
              error is an independent uniform variable of that half-width (standard deviation
              width / sqrt 3).
    """
    p = unpack(theta)
    W1, b1, W2, b2, W3 = p["W1"], p["b1"], p["W2"], p["b2"], p["W3"]
    a32 = 2.0 ** -23
    dx = u * np.abs(X) + a32 * (1.0 + np.abs(X))
    z1 = X @ W1.T + b1
    da1 = dx @ np.abs(W1).T + (u + a32) * (np.abs(X) @ np.abs(W1).T) + a32 * np.abs(b1)
    dz1 = da1 + u * (np.abs(z1) + da1)
    slope1 = 1.0 - np.tanh(np.maximum(np.abs(z1) - dz1, 0.0)) ** 2
    h1 = np.tanh(z1)
    dh1 = slope1 * dz1 + eps_t
    z2 = h1 @ W2.T + b2
    absW2 = np.abs(W2)
    da2 = dh1 @ absW2.T + (u + a32) * ((np.abs(h1) + dh1) @ absW2.T) + a32 * np.abs(b2)
    dz2 = da2 + u * (np.abs(z2) + da2)
    slope2 = 1.0 - np.tanh(np.maximum(np.abs(z2) - dz2, 0.0)) ** 2
    h2 = np.tanh(z2)
    dh2 = slope2 * dz2 + eps_t
    worst = dh2 @ np.abs(W3) + a32 * ((np.abs(h2) + dh2) @ np.abs(W3) + abs(p["b3"][0]))
    # sensitivities of y: to z2, h1, z1 and the features
    g2 = W3 * (1.0 - h2 ** 2)
    g1 = g2 @ W2
    gz1 = g1 * (1.0 - h1 ** 2)
    gx = gz1 @ W1
    r = 1.0 / 3.0  # variance of a uniform error of half-width 1
    var = (W3 ** 2).sum() * eps_t ** 2 * r * np.ones(X.shape[0])        # tanh of layer 2
    var += ((g2 * u * np.abs(z2)) ** 2).sum(1) * r                       # rounding of z2
    var += ((g2 ** 2) * ((h1 ** 2) @ ((u * absW2) ** 2).T)).sum(1) * r   # W2 in FP16
    var += ((g1 * eps_t) ** 2).sum(1) * r                                # tanh of layer 1
    var += ((gz1 * u * np.abs(z1)) ** 2).sum(1) * r                      # rounding of z1
    var += ((gz1 ** 2) * ((X ** 2) @ ((u * np.abs(W1)) ** 2).T)).sum(1) * r  # W1 in FP16
    var += ((gx * u * np.abs(X)) ** 2).sum(1) * r                        # features in FP16
    return worst, np.sqrt(var)


def test_mlp_inference_matches_oracle_forward():
    """dg_mlp_guess (FP16 tcgen05 inference) node by node against the oracle's FP64 forward pass of the
    same FP32 parameters, within the bound of FP16 operands and the FP16 hardware tanh; 37 full tiles
    of 128 nodes and a ragged tail of 45, moving gas, temperatures beyond the clamp range."""
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    mix = seeded_nasa7_mixture(7, seed=0)
    gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50)
    go = Nasa7Gas(W=mix.W, coeffs=mix.coeffs)
    rng = np.random.default_rng(8)
    theta = (glorot_params(4) + rng.normal(scale=0.1, size=N_PARAMS)).astype(np.float32)
    n = 128 * 37 + 45
    T, Y = temperature_samples(n, 7, seed=21, T_min=200.0, T_max=3300.0)
    rho = rng.uniform(0.1, 2.0, size=n)
    vel = rng.normal(scale=30.0, size=(3, n))
    q = go.conserved(rho, vel, Y, T)
    e = q[4] / q[0] - 0.5 * ((q[1:4] / q[0]) ** 2).sum(axis=0)
    norm = dict(e_mean=float(e.mean()), e_scale=float(e.std()), T_mean=1650.0, T_scale=780.0,
                T_min=1000.0, T_max=2300.0)
    dg.dg_mlp_set(gas, theta, norm)
    out = torch.empty(n, device="cuda", dtype=torch.float64)
    dg.dg_mlp_guess(gas, torch.tensor(q, device="cuda"), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    X = np.concatenate([((e - norm["e_mean"]) / norm["e_scale"])[None], q[5:] / q[0]], axis=0).T
    th64 = theta.astype(np.float64)
    y, _ = forward(th64, X)
    want = np.clip(norm["T_mean"] + norm["T_scale"] * y, norm["T_min"], norm["T_max"])
    worst, rss = _fp16_guess_error_model(th64, X)
    worst, rss = norm["T_scale"] * worst + 1e-9, norm["T_scale"] * rss  # the clamp is 1-Lipschitz
    err = np.abs(got - want)
    print(f"FP16 inference vs FP64 forward: max {err.max():.3g} K, mean {err.mean():.3g} K; "
          f"worst-case bound {worst.max():.3g} K, rss model {rss.max():.3g} K")
    assert np.all(err <= worst)
    assert np.all(err <= 4.0 * rss)   # 4 standard deviations of the independent-error model
    assert np.any(want == norm["T_min"]) and np.any(want == norm["T_max"])  # both clamps exercised
    # a weight planted in the wrong place moves the guesses far beyond the tolerance
    bad = theta.copy()
    bad[576:4672] = bad[576:4672].reshape(64, 64).T.ravel()   # W2 transposed
    y_bad, _ = forward(bad.astype(np.float64), X)
    want_bad = np.clip(norm["T_mean"] + norm["T_scale"] * y_bad, norm["T_min"], norm["T_max"])
    assert np.mean(np.abs(got - want_bad) > 4.0 * rss) > 0.5


def _train(torch, dg, n_samples=400_000, epochs=30):
    mix = seeded_nasa7_mixture(7, seed=0)
    gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50)
    T, Y = temperature_samples(n_samples, 7, seed=11)
    Td, Yd = torch.tensor(T, device="cuda"), torch.tensor(Y, device="cuda")
    e = torch.empty_like(Td)
    dg.dg_mixture_energy(gas, Td, Yd, e)
    # Newton-generated labels: solve e(T) = e from a constant seed
    q = torch.zeros((12, n_samples), device="cuda", dtype=torch.float64)
    q[0] = 1.0
    q[4] = e
    q[5:] = Yd
    Tn = torch.full_like(Td, 1650.0)
    dg.dg_temperature(gas, q, Tn)
    assert gas.status() == 0
    hist = dg.dg_mlp_train(gas, e, Yd, Tn, glorot_params(0), epochs=epochs, batch=1024, lr=3e-3, lr_decay=0.9)
    return mix, gas, hist


def _iterations(torch, dg, capi, gas, qh, seed_value=1650.0):
    n = qh.shape[1]
    q = torch.tensor(qh, device="cuda")
    it_c = torch.zeros(n, device="cuda", dtype=torch.int32)
    it_m = torch.zeros_like(it_c)
    T_c = torch.full((n,), seed_value, device="cuda", dtype=torch.float64)
    T_m = torch.empty_like(T_c)
    dg.dg_temperature(gas, q, T_c, it_c)
    dg.dg_temperature(gas, q, T_m, it_m, opts=dg._opts(t_seed=capi.DG_TSEED_MLP))
    guess = torch.empty_like(T_c)
    dg.dg_mlp_guess(gas, q, guess)
    return T_c, T_m, it_c.double().mean().item(), it_m.double().mean().item(), (guess - T_m).abs()


def test_mlp_training_reduces_loss_and_newton_iterations():
    """Trained on Newton-generated samples; on held-out samples with T spread over 300..3000 K the MLP
    seed needs fewer Newton updates than the constant seed; on the learned-form workload's field
    (which clusters near the constant seed) it does not lose.  Newton decides both: same T."""
    torch = torch_cuda()
    from paper_2512_17101_gb300 import capi, dg
    mix, gas, hist = _train(torch, dg)
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.2 * hist[0], hist
    go = Nasa7Gas(W=mix.W, coeffs=mix.coeffs)
    # held-out samples (another seed), at rest, rho = 1
    T_h, Y_h = temperature_samples(50_000, 7, seed=99)
    q_h = go.conserved(np.ones_like(T_h), np.zeros((3, T_h.size)), Y_h, T_h)
    T_c, T_m, mean_c, mean_m, gerr = _iterations(torch, dg, capi, gas, q_h)
    assert gas.status() == 0
    assert (T_c - T_m).abs().max().item() < 1e-9
    assert np.abs(T_m.cpu().numpy() - T_h).max() < 1e-8
    print(f"held-out: Newton iterations constant {mean_c:.2f}, MLP {mean_m:.2f}; "
          f"guess error mean {gerr.mean().item():.2f} K max {gerr.max().item():.1f} K")
    assert mean_m < mean_c - 0.5
    # the learned-form workload's node states (7 species, T field 300..3000 K) on a smaller box
    verts, period = box_mesh(12, 1.0)
    xyz = physical_nodes(verts, equispaced_tet_nodes(2))
    Yf, Tf, vel, p0 = mixture_primitive_state(xyz, 7, seed=0)
    rho = p0 / (go.R_mix(Yf) * Tf)
    qf = go.conserved(rho, vel, Yf, Tf).reshape(12, -1)
    T_c, T_m, mean_c, mean_m, gerr = _iterations(torch, dg, capi, gas, qf)
    assert gas.status() == 0
    assert (T_c - T_m).abs().max().item() < 1e-9
    assert np.abs(T_m.cpu().numpy() - Tf.ravel()).max() < 1e-8
    print(f"workload field: Newton iterations constant {mean_c:.2f}, MLP {mean_m:.2f}; "
          f"guess error mean {gerr.mean().item():.2f} K max {gerr.max().item():.1f} K")
    assert mean_m <= mean_c + 0.2
