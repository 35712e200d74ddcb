"""Batched engine (many 2D constant-medium problems per launch) against the
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
    # a varying medium is not batchable: create refuses, the batched solve runs instance by instance
    wv = custom((64, 64), 80, 8, True, 9, seed=31, family=4, levels=2)
    pv, wave_v, wav_v = make_pair(wv)
    with pytest.raises(_lib.PatError):
        _lib.pat_batch_create([plans[0].handle, pv.handle])
    y2 = [ys[0], torch.as_tensor(wave_v.forward(wv.x_true), dtype=torch.float32, device="cuda")]
    x2 = [torch.empty(ws[0].shape, device="cuda"), torch.empty(wv.shape, device="cuda")]
    rc, per = _lib.pat_solve_batched([plans[0].handle, pv.handle], y2, [1e-2, 1e-2], [1.0, 1.0], 6, x2)
    assert rc == 0 and per == [0, 0]
    _, xr, _ = oracle.cg(wave_v, wav_v, y2[1].cpu().numpy().astype(np.float64), 1e-2, 1.0, 6)
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


def test_batch_64_uneven_instances_sampled():
    """64 instances, n in {128, ..., 512}, nt = ceil(sqrt(2) n / 0.3), order 8,
    64-512 sensors on circles or arcs: batched K against the oracle on the
    smallest and the largest instance, batched K* of the noisy data on the
    largest, 50-iteration batched solve against
    pat_solve on three instances and against the oracle's CG on the smallest."""
    torch = need_gpu()
    from paper_2507_02401_gb300 import Batch
    ws = synth.batched_workloads()
    plans = [make_pair(w)[0] for w in ws]
    batch = Batch(plans)
    ys = batch.forward([w.x_true for w in ws])
    small = min(range(len(ws)), key=lambda i: ws[i].N)
    large = max(range(len(ws)), key=lambda i: ws[i].N)
    for i in (small, large):
        w = ws[i]
        wave = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors)
        assert rel(ys[i].cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    rng = np.random.default_rng(9)
    data = [synth.add_noise(y.cpu().numpy().astype(np.float64), w.noise, rng) for y, w in zip(ys, ws)]
    # batched K* of the noisy data on the largest instance (512^2, 2414 steps)
    w = ws[large]
    wave = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors)
    assert rel(batch.adjoint(data)[large].cpu().numpy(), wave.adjoint(data[large])) <= TOL_OP
    ss = [w.s[0] for w in ws]
    # alpha relative to lambda_max of E_s* K* K E_s (power iteration through the batch)
    g = torch.Generator(device="cuda").manual_seed(0)
    vs = [torch.randn(p.N, device="cuda", generator=g) for p in plans]
    vs = [v / v.norm() for v in vs]
    for _ in range(8):
        hs = batch.adjoint(batch.forward([p.Es(v, s) for p, v, s in zip(plans, vs, ss)]))
        hv = [p.EsT(h, s) for p, h, s in zip(plans, hs, ss)]
        lams = [float(h.norm()) for h in hv]
        vs = [h / lam for h, lam in zip(hv, lams)]
    alphas = [w.alpha[0] * lam for w, lam in zip(ws, lams)]
    xs, rc, per = batch.solve(data, alphas, ss, 50)
    assert rc == 0 and per == [0] * len(ws)
    for i in (small, len(ws) // 2, large):
        _, x1, _ = plans[i].solve(data[i], alphas[i], ss[i], 50)
        assert rel(xs[i].cpu().numpy(), x1.cpu().numpy()) <= 1e-4
    w = ws[small]
    wave = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors)
    wav = oracle.Wavelet(w.shape, w.family, w.levels)
    _, x_ref, _ = oracle.cg(wave, wav, data[small], alphas[small], ss[small], 50)
    assert rel(xs[small].cpu().numpy(), x_ref) <= TOL_X
    torch.cuda.synchronize()
