"""Batched engine (many 2D problems per launch, constant or varying medium) against the
FP64 oracle per instance: K and K* (relative L2 <= 1e-5), both tile heights
the autotuner chooses between, the CG solve (<= 1e-4 on the final image),
pat_solve_batched routing and fallback, validation, the autograd wrapper,
and the 64-instance workload of uneven size (sampled instances)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5
TOL_X = 1e-4

# shape (ny, nx), nt, order, ns, levels: uneven sizes, nt and sensor counts
SMALL = [((64, 64), 150, 8, 20, 3), ((96, 128), 220, 8, 33, 2), ((128, 72), 90, 8, 7, 3),
         ((70, 136), 260, 8, 40, 1), ((40, 40), 60, 8, 5, 3), ((8, 16), 30, 8, 2, 0)]


def small_batch(seed=0):
    ws = [custom(shape, nt, order, False, ns, seed=seed + i, family=4 if levels else 2, levels=levels)
          for i, (shape, nt, order, ns, levels) in enumerate(SMALL)]
    pairs = [make_pair(w) for w in ws]
    return ws, pairs


@pytest.mark.parametrize("tile_y", ["64", "32", None])
def test_batch_forward_adjoint_parity(monkeypatch, tile_y):
    need_gpu()
    from paper_2507_02401_gb300 import Batch
    if tile_y:
        monkeypatch.setenv("PAT_BATCH_TILE_Y", tile_y)
    ws, pairs = small_batch()
    batch = Batch([p for p, _, _ in pairs])
    if tile_y:
        assert batch.info["tile_rows"] == int(tile_y)
    ys = batch.forward([w.x_true for w in ws])
    for w, (_, wave, _), y in zip(ws, pairs, ys):
        assert rel(y.cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    rng = np.random.default_rng(4)
    rs = [rng.standard_normal((w.ns, w.nt)) for w in ws]
    xs = batch.adjoint(rs)
    for r, (_, wave, _), x in zip(rs, pairs, xs):
        assert rel(x.cpu().numpy(), wave.adjoint(r)) <= TOL_OP


def test_batch_matches_single_instance_engines():
    need_gpu()
    from paper_2507_02401_gb300 import Batch
    ws, pairs = small_batch(seed=10)
    batch = Batch([p for p, _, _ in pairs])
    ys = batch.forward([w.x_true for w in ws])
    for w, (plan, _, _), y in zip(ws, pairs, ys):
        assert rel(y.cpu().numpy(), plan.forward(w.x_true).cpu().numpy()) <= 2e-6


def test_batch_solve_against_oracle_cg():
    need_gpu()
    from paper_2507_02401_gb300 import Batch
    ws, pairs = small_batch(seed=20)
    rng = np.random.default_rng(5)
    ys = [synth.add_noise(wave.forward(w.x_true), 0.01, rng) for w, (_, wave, _) in zip(ws, pairs)]
    alphas = [10.0 ** rng.uniform(-3, -1) for _ in ws]
    ss = [float(rng.choice([1.0, 1.5, 2.0])) for _ in ws]
    batch = Batch([p for p, _, _ in pairs])
    iters = 12
    xs, rc, per = batch.solve(ys, alphas, ss, iters)
    assert rc == 0 and per == [0] * len(ws)
    assert batch.info["graph_nodes"] > 0
    for w, (_, wave, wav), y, a, s, x in zip(ws, pairs, ys, alphas, ss, xs):
        _, x_ref, _ = oracle.cg(wave, wav, y, a, s, iters)
        assert rel(x.cpu().numpy(), x_ref) <= TOL_X
    # a second solve with other alphas re-captures the graph and still agrees
    alphas2 = [a * 3.0 for a in alphas]
    xs2, rc2, _ = batch.solve(ys, alphas2, ss, iters)
    assert rc2 == 0
    w, (_, wave, wav), y = ws[1], pairs[1], ys[1]
    _, x_ref, _ = oracle.cg(wave, wav, y, alphas2[1], ss[1], iters)
    assert rel(xs2[1].cpu().numpy(), x_ref) <= TOL_X


def test_solve_batched_routes_and_falls_back():
    torch = need_gpu()
    from paper_2507_02401_gb300 import _lib
    ws, pairs = small_batch(seed=30)
    plans = [p for p, _, _ in pairs]
    rng = np.random.default_rng(6)
    ys = [torch.as_tensor(wave.forward(w.x_true), dtype=torch.float32, device="cuda")
          for w, (_, wave, _) in zip(ws, pairs)]
    alphas = [1e-2] * len(ws)
    ss = [1.0] * len(ws)
    xs = [torch.empty(w.shape, device="cuda") for w in ws]
    rc, per = _lib.pat_solve_batched([p.handle for p in plans], ys, alphas, ss, 6, xs)
    assert rc == 0 and per == [0] * len(ws)
    for p, y, a, s, x in zip(plans, ys, alphas, ss, xs):
        _, x1, _ = p.solve(y, a, s, 6)  # another engine: held to the solve bound
        assert rel(x.cpu().numpy(), x1.cpu().numpy()) <= TOL_X
    # a varying medium batches with constant ones; another stencil order is not batchable: create
    # refuses and the batched solve runs instance by instance
    wv = custom((64, 64), 80, 8, True, 9, seed=31, family=4, levels=2)
    pv, wave_v, wav_v = make_pair(wv)
    w4 = custom((64, 64), 80, 4, False, 9, seed=32, family=4, levels=2)
    p4, wave_4, wav_4 = make_pair(w4)
    with pytest.raises(_lib.PatError):
        _lib.pat_batch_create([plans[0].handle, p4.handle])
    for pb, wave_b, wav_b, wb in ((pv, wave_v, wav_v, wv), (p4, wave_4, wav_4, w4)):
        y2 = [ys[0], torch.as_tensor(wave_b.forward(wb.x_true), dtype=torch.float32, device="cuda")]
        x2 = [torch.empty(ws[0].shape, device="cuda"), torch.empty(wb.shape, device="cuda")]
        rc, per = _lib.pat_solve_batched([plans[0].handle, pb.handle], y2, [1e-2, 1e-2], [1.0, 1.0], 6, x2)
        assert rc == 0 and per == [0, 0]
        _, xr, _ = oracle.cg(wave_b, wav_b, y2[1].cpu().numpy().astype(np.float64), 1e-2, 1.0, 6)
        assert rel(x2[1].cpu().numpy(), xr) <= TOL_X


def test_batch_validation():
    need_gpu()
    from paper_2507_02401_gb300 import _lib
    ws, pairs = small_batch(seed=40)
    h = pairs[0][0].handle
    with pytest.raises(_lib.PatError):
        _lib.pat_batch_create([h, h])  # one plan twice
    w2 = custom((64, 64), 80, 4, False, 9, seed=41)
    p2, _, _ = make_pair(w2)
    with pytest.raises(_lib.PatError):
        _lib.pat_batch_create([h, p2.handle])  # different stencil order
    w3 = custom((64, 66), 80, 8, False, 9, seed=42)
    p3, _, _ = make_pair(w3)
    with pytest.raises(_lib.PatError):
        _lib.pat_batch_create([p3.handle])  # nx not divisible by 4


def test_batch_autograd_dot_product():
    torch = need_gpu()
    from paper_2507_02401_gb300 import Batch
    from paper_2507_02401_gb300.autograd import batch_K
    ws, pairs = small_batch(seed=50)
    batch = Batch([p for p, _, _ in pairs])
    rng = np.random.default_rng(8)
    xs = [torch.tensor(rng.standard_normal(w.shape), dtype=torch.float32, device="cuda", requires_grad=True)
          for w in ws]
    vs = [torch.tensor(rng.standard_normal((w.ns, w.nt)), dtype=torch.float32, device="cuda") for w in ws]
    ys = batch_K(batch, xs)
    loss = sum((y.double() * v.double()).sum() for y, v in zip(ys, vs))
    loss.backward()
    for x, v, (_, wave, _), w in zip(xs, vs, pairs, ws):
        ref = wave.adjoint(v.cpu().numpy().astype(np.float64))
        assert rel(x.grad.cpu().numpy(), ref) <= TOL_OP


def _oracle_lambda_max(wave, wav, s, iters=15, seed=0):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(wave.N)
    v /= np.linalg.norm(v)
    H = oracle.normal_op(wave, wav, s, 0.0)
    lam = 0.0
    for _ in range(iters):
        hv = H(v)
        lam = float(np.linalg.norm(hv))
        v = hv / lam
    return lam


# three 128^2 instances of the 64-instance workload spanning its conditioning: alpha_rel 1.1e-4
# (s = 1.5), 8.2e-4 (s = 1.5), 7.1e-2 (s = 1)
COMPARED = (61, 31, 11)


def test_batch_64_uneven_instances_sampled():
    """64 instances, n in {128, ..., 512}, nt = ceil(sqrt(2) n / 0.3), order 8,
    64-512 sensors on circles or arcs.  Batched K against the oracle on the
    smallest and the largest instance; batched K* of noisy data simulated by
    the oracle on the largest (512^2, 2414 steps); the 50-iteration batched
    solve against pat_solve on three instances and, on three 128^2 instances
    spanning the conditioning, against the oracle's CG (oracle data, oracle
    lambda_max).  Accuracy bound per reading A14: <= 1e-4 against the
    oracle's 50-step image where alpha_rel >= 1e-2; below that, as accurate
    as the oracle's 50-step image against the oracle's converged minimiser
    (within 10 % of the oracle's own distance) and within 2e-2 of its 50-step
    image (CG after 50 steps at this conditioning is far from converged and
    shifts with any rounding; measured up to 7.9e-3 at alpha_rel 1.1e-4)."""
    torch = need_gpu()
    from paper_2507_02401_gb300 import Batch
    ws = synth.batched_workloads()
    plans = [make_pair(w)[0] for w in ws]
    batch = Batch(plans)
    ys = batch.forward([w.x_true for w in ws])
    small = min(range(len(ws)), key=lambda i: ws[i].N)
    large = max(range(len(ws)), key=lambda i: ws[i].N)
    waves = {}
    for i in set((small, large) + COMPARED):
        w = ws[i]
        waves[i] = (oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors),
                    oracle.Wavelet(w.shape, w.family, w.levels))
    y_or = {i: waves[i][0].forward(ws[i].x_true) for i in waves}
    for i in (small, large):
        assert rel(ys[i].cpu().numpy(), y_or[i]) <= TOL_OP
    rng = np.random.default_rng(9)
    # data: GPU-simulated for the instances not compared with the oracle, oracle-simulated for the others
    data = [synth.add_noise(y_or[i] if i in y_or else ys[i].cpu().numpy().astype(np.float64), w.noise, rng)
            for i, w in enumerate(ws)]
    assert rel(batch.adjoint(data)[large].cpu().numpy(), waves[large][0].adjoint(data[large])) <= TOL_OP
    ss = [w.s[0] for w in ws]
    # alpha relative to lambda_max of E_s* K* K E_s: the oracle's for the compared instances, a power
    # iteration through the batch for the others
    g = torch.Generator(device="cuda").manual_seed(0)
    vs = [torch.randn(p.N, device="cuda", generator=g) for p in plans]
    vs = [v / v.norm() for v in vs]
    for _ in range(8):
        hs = batch.adjoint(batch.forward([p.Es(v, s) for p, v, s in zip(plans, vs, ss)]))
        hv = [p.EsT(h, s) for p, h, s in zip(plans, hs, ss)]
        lams = [float(h.norm()) for h in hv]
        vs = [h / lam for h, lam in zip(hv, lams)]
    for i in COMPARED:
        lams[i] = _oracle_lambda_max(waves[i][0], waves[i][1], ss[i])
    alphas = [w.alpha[0] * lam for w, lam in zip(ws, lams)]
    xs, rc, per = batch.solve(data, alphas, ss, 50)
    assert rc == 0 and per == [0] * len(ws)
    for i in (small, len(ws) // 2, large):
        _, x1, _ = plans[i].solve(data[i], alphas[i], ss[i], 50)
        d = rel(xs[i].cpu().numpy(), x1.cpu().numpy())
        print(f"instance {i} (alpha_rel {ws[i].alpha[0]:.2e}): batched vs pat_solve {d:.2e}")
        if ws[i].alpha[0] >= 1e-2:  # two FP32 engines: the same bound as against the oracle
            assert d <= TOL_X
    for i in COMPARED:
        wave, wav = waves[i]
        xb = xs[i].cpu().numpy()
        _, x50, _ = oracle.cg(wave, wav, data[i], alphas[i], ss[i], 50)
        e50 = rel(xb, x50)
        print(f"instance {i} (alpha_rel {ws[i].alpha[0]:.2e}, s {ss[i]}): batched vs oracle CG-50 {e50:.2e}")
        if ws[i].alpha[0] >= 1e-2:
            assert e50 <= TOL_X
            continue
        _, x_c, k, rr = oracle.cg_converged(wave, wav, data[i], alphas[i], ss[i], rtol=1e-9)
        e_gpu, e_ora = rel(xb, x_c), rel(x50, x_c)
        print(f"   against the converged minimiser ({k} steps): batched {e_gpu:.3e}, oracle CG-50 {e_ora:.3e}")
        assert abs(e_gpu - e_ora) <= 0.1 * e_ora
        assert e50 <= 2e-2
    torch.cuda.synchronize()


@pytest.mark.parametrize("launch", [1, 2], ids=["per-step", "one-launch"])
def test_batch_varying_media_and_launch_forms(launch):
    """Constant and varying media in one batch (kappa per cell read by the
    batched kernel), in both launch forms: K and K* against the oracle
    (K* of noisy data simulated by the oracle) and a 10-iteration solve."""
    need_gpu()
    from paper_2507_02401_gb300 import Batch
    shapes = [((64, 96), True), ((96, 64), False), ((128, 128), True), ((40, 72), True)]
    ws = [custom(sh, 180 + 40 * i, 8, varc, 11 + 3 * i, seed=60 + i, family=4, levels=2)
          for i, (sh, varc) in enumerate(shapes)]
    pairs = [make_pair(w) for w in ws]
    batch = Batch([p for p, _, _ in pairs])
    batch.set_launch(launch)
    assert batch.info["launch"] == ("one per step" if launch == 1 else "one per application")
    ys = batch.forward([w.x_true for w in ws])
    rng = np.random.default_rng(61)
    data = []
    for w, (_, wave, _), y in zip(ws, pairs, ys):
        yo = wave.forward(w.x_true)
        assert rel(y.cpu().numpy(), yo) <= TOL_OP
        data.append(synth.add_noise(yo, 0.02, rng))
    xs = batch.adjoint(data)
    for (_, wave, _), x, d in zip(pairs, xs, data):
        assert rel(x.cpu().numpy(), wave.adjoint(d)) <= TOL_OP
    alphas = [1e-2, 3e-2, 2e-2, 5e-2]
    ss = [1.0, 1.5, 2.0, 1.0]
    xs, rc, per = batch.solve(data, alphas, ss, 10)
    assert rc == 0 and per == [0] * len(ws)
    for (_, wave, wav), x, d, a, s in zip(pairs, xs, data, alphas, ss):
        _, x_ref, _ = oracle.cg(wave, wav, d, a, s, 10)
        assert rel(x.cpu().numpy(), x_ref) <= TOL_X

