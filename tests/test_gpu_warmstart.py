"""Learned warm start: feature/target geometry against a numpy restatement of
their definitions, and the gain of a network trained on the solver's own
star-robot trajectories over the extrapolated Newton guess."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_2311_18126_gb300 import dismech
    return dismech


def _rod_offsets(npr):
    off = np.zeros(len(npr) + 1, np.int64)
    off[1:] = np.cumsum(4 * np.asarray(npr) - 1)
    return off


def _expected(desc, params, q, v, d1, kbar_slots, npr, vprev):
    """Features [S, 64] and extrapolated guesses, from the documented
    definitions (segments: rods in order, nodes i = 1..N-1)."""
    dt = params["dt"]
    g = np.asarray(params["g"])
    off = _rod_offsets(npr)
    lbar = 0.1 / (npr[0] - 1)  # star robots: uniform spacing
    feats, guess, basis, sigmas = [], [], [], []
    e0 = 0
    k0 = 0
    for r, N in enumerate(npr):
        Q = q[off[r]:off[r + 1]]
        V = v[off[r]:off[r + 1]]
        X = lambda j: Q[4 * j:4 * j + 3]
        XV = lambda j: V[4 * j:4 * j + 3]
        for i in range(1, N):
            e = e0 + i - 1
            t = X(i) - X(i - 1)
            t = t / np.linalg.norm(t)
            a = d1[e]
            b = np.cross(t, a)
            B = np.stack([t, a, b])
            f = np.zeros(64)
            for w, j in enumerate(range(i - 2, i + 3)):
                if 0 <= j < N:
                    f[6 * w:6 * w + 3] = B @ (X(j) - X(i)) / lbar
                    f[6 * w + 3:6 * w + 6] = B @ (dt * XV(j)) / lbar
                    f[30 + w] = 1.0
            for w, ee in enumerate(range(i - 2, i + 1)):
                if 0 <= ee <= N - 2:
                    f[35 + w] = dt * V[4 * ee + 3]
                    if w != 1:
                        f[38 + (w == 2)] = Q[4 * ee + 3] - Q[4 * (i - 1) + 3]
            for w, m in enumerate(range(i - 1, i + 2)):
                if 1 <= m <= N - 2:
                    f[40 + 2 * w:42 + 2 * w] = kbar_slots[k0 + m - 1]
            f[46:49] = B @ (g * dt * dt) / lbar
            h = desc["radius"][r]
            f[49] = np.clip((X(i)[2] - params["ground_z"]) / h, -5.0, 20.0)
            f[50] = desc["ground_mu"][r]
            f[51] = np.log10(desc["E"][r])
            f[52] = np.log10(h / lbar)
            f[53] = np.log10(desc["rho"][r])
            # the previous step's correction dt (qdot_n - qdot_{n-1}),
            # relative to the segment's scales
            VP = vprev[off[r]:off[r + 1]]
            pc = B @ (dt * (XV(i) - VP[4 * i:4 * i + 3])) / lbar
            pth = dt * (V[4 * (i - 1) + 3] - VP[4 * (i - 1) + 3])
            sig = max(np.linalg.norm(pc), np.linalg.norm(g) * dt * dt / lbar)
            sth = max(abs(pth), 1e-9)
            f[55:58] = pc / sig
            f[58] = pth / sth
            f[59] = np.log10(sig)
            f[60] = np.log10(sth)
            sigmas.append((sig, sth))
            feats.append(f)
            guess.append(np.concatenate([X(i) + dt * XV(i),
                                         [Q[4 * (i - 1) + 3] + dt * V[4 * (i - 1) + 3]]]))
            basis.append(B)
        e0 += N - 1
        k0 += N - 2
    return np.array(feats), np.array(guess), np.array(basis), lbar, np.array(sigmas)


def test_features_and_targets_match_definitions():
    dmx = _lib()
    desc, params, gait = workloads.star_robots(n_robots=3, seed=5, nodes_per_limb=8)
    sys = dmx.System(desc, params)
    npr = list(desc["nodes_per_rod"])
    dt = params["dt"]
    S = sys.ws_enable()
    assert S == sum(n - 1 for n in npr)
    for k in range(4):
        sys.set_natural_curvature(0, sys.n_rods, workloads.gait_kbar(gait, k * dt))
        vprev = sys.get_state()[1]
        sys.step(1)
    kb = workloads.gait_kbar(gait, 4 * dt)
    sys.set_natural_curvature(0, sys.n_rods, kb)
    q, v = sys.get_state()
    d1, _ = sys.get_frames()
    feat = torch.zeros((S, 64), dtype=torch.float32, device="cuda")
    tgt = torch.zeros((S, 4), dtype=torch.float32, device="cuda")
    sys.ws_capture_features(feat)
    sys.step(1)
    sys.ws_capture_targets(tgt)
    torch.cuda.synchronize()
    F = feat.cpu().numpy().astype(np.float64)
    T = tgt.cpu().numpy().astype(np.float64)
    ef, guess, B, lbar, sig = _expected(desc, params, q, v, d1, kb, npr, vprev)
    cols = list(range(0, 54))
    np.testing.assert_allclose(F[:, cols], ef[:, cols], rtol=2e-6, atol=2e-6)
    assert np.abs(ef[:, 55:59]).max() > 0.5
    np.testing.assert_allclose(F[:, 55:61], ef[:, 55:61], rtol=1e-5, atol=1e-5)
    assert np.all(F[:, 61:] == 0.0)
    # targets: local-frame correction of the guess, rebuilt from q_{n+1}
    q1, _ = sys.get_state()
    off = _rod_offsets(npr)
    want = []
    for r, N in enumerate(npr):
        Q = q1[off[r]:off[r + 1]]
        for i in range(1, N):
            want.append(np.concatenate([Q[4 * i:4 * i + 3], [Q[4 * (i - 1) + 3]]]))
    want = np.array(want)
    dx = want[:, :3] - guess[:, :3]
    loc = np.einsum("sij,sj->si", B, dx) / lbar / sig[:, :1]
    np.testing.assert_allclose(T[:, :3], loc, rtol=1e-5, atol=1e-7 * np.abs(loc).max())
    tw = (want[:, 3] - guess[:, 3]) / sig[:, 1]
    np.testing.assert_allclose(T[:, 3], tw, rtol=1e-5, atol=1e-7 * np.abs(tw).max())
    assert np.abs(loc).max() > 0.0


def test_learned_warm_start_against_extrapolation():
    """Trains the network on solver-generated star-robot trajectories and
    deploys it on unseen robots next to the plain method: both reach the
    same tolerance and the same trajectory; the iteration counts and wall
    times of both are printed (the measured gain of the learned guess).
    The merit test keeps a learned guess only where it lowers the residual
    of the extrapolation, so the learned run cannot take many more Newton
    iterations than the plain one."""
    dmx = _lib()
    from paper_2311_18126_gb300 import warmstart as ws
    desc, params, gait = workloads.star_robots(n_robots=64, seed=21)
    dt = params["dt"]
    train_sys = dmx.System(desc, params)
    feats, tgts = ws.collect(train_sys, 240,
                             controls=lambda k: workloads.gait_kbar(gait, k * dt))
    train_sys.close()
    mlp, norm, losses = ws.train(feats, tgts, iters=1500, batch=8192, lr=1e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0]
    del feats, tgts
    # unseen robots: seeded limb counts and gaits differ from training
    desc2, params2, gait2 = workloads.star_robots(n_robots=32, seed=77)
    ctl = lambda k: workloads.gait_kbar(gait2, k * dt)
    plain = dmx.System(desc2, params2)
    learned = dmx.System(desc2, params2)
    it_p, wall_p, res_p = ws.run(plain, 80, controls=ctl)
    it_l, wall_l, res_l = ws.run(learned, 80, controls=ctl, mlp=mlp, norm=norm)
    assert np.all(res_p <= params2["tol"]) and np.all(res_l <= params2["tol"])
    mean_p, mean_l = it_p[5:].mean(), it_l[5:].mean()
    print("iterations/step: extrapolation %.3f learned %.3f; slowest robot per step: "
          "%.2f vs %.2f; wall %.3f s vs %.3f s" % (mean_p, mean_l, it_p[5:].max(1).mean(),
                                                    it_l[5:].max(1).mean(), wall_p, wall_l))
    assert mean_l <= 1.25 * mean_p
    qp, _ = plain.get_state()
    ql, _ = learned.get_state()
    scale = np.abs(qp).max()
    assert np.abs(qp - ql).max() <= 1e-5 * scale
