"""Batched plans (many independent transforms in one plan and one CUDA graph).

* every transform of a batch against the plain oracle (E_i <= eps_i);
* a batched plan returns exactly what separate single plans return (the same
  kernels run the same per-band work, only grouped into shared launches);
* the batched workload of 512 transforms with log-uniform degrees
  N_i = floor(2^U), U ~ U[8, 16], M_i = N_i, disk-uniform nodes, on a seeded
  sample of transforms;
* CUDA-graph replay: repeated and re-targeted executes give the same results;
* shared node sets (one node array for every transform, sorted once per
  distinct N_i, weight tables shared by transforms of equal N_i): each
  transform against the oracle, and bitwise equal to the same batch planned
  with the node set repeated per transform;
* the autotuner's choices (route bias, oversampling, fused gather, grids per
  launch) stay within the accuracy bound and are reused from its cache.
"""
import numpy as np
import pytest

import oracle
from paper_1606_03255_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def fl():
    from paper_1606_03255_gb300 import build as libbuild
    libbuild.build()
    from paper_1606_03255_gb300 import fl as flmod
    flmod.load()
    return flmod


def _tol(eps, prec, ref, c):
    if prec == "fp64":
        return eps
    return eps + 32 * U32 * np.max(np.abs(ref)) / np.sum(np.abs(c))


def _batch(Ns, Ms, seed, kinds=("disk",)):
    cs, ws = [], []
    for i, (N, M) in enumerate(zip(Ns, Ms)):
        cs.append(W.coefficients(N, seed=seed + i))
        kind = kinds[i % len(kinds)]
        w = (W.nodes_disk_uniform(M, seed=seed + 1000 + i) if kind == "disk"
             else W.nodes_circle_clustered(M, seed=seed + 1000 + i))
        ws.append(w)
    return cs, ws


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("route", ["auto", "nfft"])
def test_batch_against_oracle(fl, prec, eps, route):
    Ns = [1, 300, 5000, 20000, 777, 4096, 64, 12345]
    Ms = [7, 250, 3000, 2000, 0, 4096, 100, 1500]
    cs, ws = _batch(Ns, Ms, seed=10, kinds=("disk", "clustered"))
    ws[2] = np.concatenate([ws[2][:-1], [[0.25, 6.0]]])      # a Z^0 node
    dev = torch.device("cuda")
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    plan = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), eps,
                          precision=prec, route=route)
    assert plan.info()["batch"] == len(Ns)
    f = plan.execute(torch.from_numpy(np.concatenate(cs)).to(cdt).to(dev))
    torch.cuda.synchronize()
    f = f.cpu().numpy().astype(np.complex128)
    moff = 0
    for c, w, M in zip(cs, ws, Ms):
        if M:
            ref = oracle.flt_direct(c, w)
            E = oracle.error_E(ref, f[moff:moff + M], c)
            assert E <= _tol(eps, prec, ref, c), (len(c), M, E)
        moff += M
    plan.close()


def test_batch_equals_separate_plans(fl):
    Ns = [2000, 50000, 300, 9000]
    Ms = [1000, 4000, 300, 2500]
    cs, ws = _batch(Ns, Ms, seed=20, kinds=("clustered", "disk"))
    dev = torch.device("cuda")
    bp = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), 1e-6)
    fb = bp.execute(torch.from_numpy(np.concatenate(cs)).to(torch.complex64).to(dev)).cpu().numpy()
    moff = 0
    for c, w, M in zip(cs, ws, Ms):
        sp = fl.Plan(len(c), torch.from_numpy(w).to(dev), 1e-6)
        fs = sp.execute(torch.from_numpy(c).to(torch.complex64).to(dev)).cpu().numpy()
        assert np.array_equal(fs, fb[moff:moff + M])
        moff += M
        sp.close()
    bp.close()


def test_batched_workload_512_sampled(fl):
    Ns = W.batched_degrees(512, seed=0)
    Ms = Ns.copy()
    rng = np.random.default_rng(1)
    dev = torch.device("cuda")
    cs = [W.coefficients(int(N), seed=2 + i).astype(np.complex64) for i, N in enumerate(Ns)]
    ws = [W.nodes_disk_uniform(int(M), seed=5000 + i) for i, M in enumerate(Ms)]
    plan = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), 1e-6)
    f = plan.execute(torch.from_numpy(np.concatenate(cs)).to(dev)).cpu().numpy()
    moff = np.concatenate([[0], np.cumsum(Ms)])
    for i in sorted(rng.choice(512, 24, replace=False)):
        c = cs[i].astype(np.complex128)
        idx = rng.choice(int(Ms[i]), min(int(Ms[i]), 128), replace=False)
        ref = oracle.flt_direct(c, ws[i][idx])
        got = f[moff[i]:moff[i + 1]][idx].astype(np.complex128)
        assert oracle.error_E(ref, got, c) <= _tol(1e-6, "fp32", ref, c), i
    plan.close()


def test_graph_replay_and_retarget(fl):
    Ns, Ms = [3000, 700], [2000, 900]
    cs, ws = _batch(Ns, Ms, seed=30)
    dev = torch.device("cuda")
    plan = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), 1e-6)
    c = torch.from_numpy(np.concatenate(cs)).to(torch.complex64).to(dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        f1 = plan.execute(c)
        f2 = plan.execute(c)                    # replayed graph
        out = torch.empty_like(f1)
        plan.execute(c, out=out)                # new buffer: captured again
        c2 = c * 2
        f3 = plan.execute(c2)
    s.synchronize()
    assert torch.equal(f1, f2) and torch.equal(f1, out)
    assert torch.allclose(f3, 2 * f1, rtol=1e-5, atol=1e-3)
    # single plans with graph replay give the same result as plain launches
    sp_g = fl.Plan(Ns[0], torch.from_numpy(ws[0]).to(dev), 1e-6, use_graph=True)
    sp_p = fl.Plan(Ns[0], torch.from_numpy(ws[0]).to(dev), 1e-6, use_graph=False)
    c0 = torch.from_numpy(cs[0]).to(torch.complex64).to(dev)
    with torch.cuda.stream(s):
        a = sp_g.execute(c0)
        a2 = sp_g.execute(c0)
        b = sp_p.execute(c0)
    s.synchronize()
    assert torch.equal(a, b) and torch.equal(a, a2)
    plan.close()
    sp_g.close()
    sp_p.close()


def test_batched_is_forward_only(fl):
    Ns, Ms = [100, 200], [50, 60]
    cs, ws = _batch(Ns, Ms, seed=40)
    dev = torch.device("cuda")
    plan = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), 1e-6)
    r = torch.zeros(sum(Ms), dtype=torch.complex64, device=dev)
    out = torch.zeros(sum(Ns), dtype=torch.complex64, device=dev)
    st = fl.fl_adjoint(plan.handle, r.data_ptr(), out.data_ptr(), None)
    assert st == fl.FL_EUNSUPPORTED
    plan.close()


def test_autotuned_plans(fl):
    # the autotuner keeps the fastest route bias; results stay within the bound
    Ns = W.batched_degrees(32, seed=3)
    cs, ws = _batch(Ns, Ns, seed=50)
    dev = torch.device("cuda")
    nodes = torch.from_numpy(np.concatenate(ws)).to(dev)
    plan = fl.BatchedPlan(Ns, Ns, nodes, 1e-6, autotune=True)
    inf = plan.info()
    bias = inf["direct_bias"]
    assert bias in (0.125, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0)
    assert inf["autotuned"] and inf["oversampling"] in ("auto", "2")
    assert inf["fuse_gather"] in ("auto", "off") and inf["rhs_per_launch"] in (0, 12, 36)
    f = plan.execute(torch.from_numpy(np.concatenate(cs)).to(torch.complex64).to(dev)).cpu().numpy()
    moff = 0
    for c, w, M in zip(cs, ws, Ns):
        idx = np.arange(0, M, max(1, M // 64))
        ref = oracle.flt_direct(c, w[idx])
        assert oracle.error_E(ref, f[moff:moff + M][idx], c) <= _tol(1e-6, "fp32", ref, c)
        moff += M
    # the same workload again: the cached choice is reused
    plan2 = fl.BatchedPlan(Ns, Ns, nodes, 1e-6, autotune=True)
    inf2 = plan2.info()
    for k in ("direct_bias", "oversampling", "fuse_gather", "rhs_per_launch"):
        assert inf2[k] == inf[k], k
    single = fl.Plan(int(Ns[0]), torch.from_numpy(ws[0]).to(dev), 1e-6, autotune=True)
    fs = single.execute(torch.from_numpy(cs[0]).to(torch.complex64).to(dev)).cpu().numpy()
    ref = oracle.flt_direct(cs[0], ws[0])
    assert oracle.error_E(ref, fs, cs[0]) <= _tol(1e-6, "fp32", ref, cs[0])
    for p in (plan, plan2, single):
        p.close()


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_shared_nodes(fl, prec, eps):
    # six transforms on one node set, three distinct N (grids from 2^9 to 2^16
    # points, fused and split bands in FP32); nodes of both distributions and a
    # Z^0 node
    Ns = [20000, 5000, 20000, 300, 5000, 20000]
    M = 3000
    w = np.concatenate([W.nodes_circle_clustered(M // 2, seed=61),
                        W.nodes_disk_uniform(M - M // 2 - 1, seed=62), [[0.4, 7.0]]])
    cs = [W.coefficients(N, seed=70 + i) for i, N in enumerate(Ns)]
    dev = torch.device("cuda")
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    c = torch.from_numpy(np.concatenate(cs)).to(cdt).to(dev)
    shared = fl.BatchedPlan(Ns, None, torch.from_numpy(w).to(dev), eps, precision=prec,
                            shared_nodes=True)
    rep = fl.BatchedPlan(Ns, [M] * len(Ns), torch.from_numpy(np.concatenate([w] * len(Ns))).to(dev),
                         eps, precision=prec)
    fs = shared.execute(c)
    fr = rep.execute(c)
    torch.cuda.synchronize()
    inf_s, inf_r = shared.info(), rep.info()
    assert inf_s["batch"] == len(Ns) and inf_s["M"] == M * len(Ns)
    # one weight table per distinct N
    assert inf_s["scratch_bytes"] < inf_r["scratch_bytes"]
    fs = fs.cpu().numpy()
    assert np.array_equal(fs, fr.cpu().numpy())
    fs = fs.astype(np.complex128)
    for i, N in enumerate(Ns):
        ref = oracle.flt_direct(cs[i], w)
        E = oracle.error_E(ref, fs[i * M:(i + 1) * M], cs[i])
        assert E <= _tol(eps, prec, ref, cs[i]), (i, N, E)
    shared.close()
    rep.close()


def test_shared_nodes_edge_cases(fl):
    dev = torch.device("cuda")
    # an empty shared node set: nothing to evaluate
    bp = fl.BatchedPlan([100, 200], None, torch.zeros((0, 2), dtype=torch.float64, device=dev), 1e-6,
                        shared_nodes=True)
    assert bp.info()["M"] == 0
    f = bp.execute(torch.zeros(300, dtype=torch.complex64, device=dev))
    assert f.numel() == 0
    bp.close()
    # one transform, and several of one size: the same as a single plan
    w = W.nodes_disk_uniform(700, seed=81)
    c = W.coefficients(5000, seed=82)
    sp = fl.Plan(5000, torch.from_numpy(w).to(dev), 1e-6)
    ref = sp.execute(torch.from_numpy(c).to(torch.complex64).to(dev)).cpu().numpy()
    sp.close()
    for B in (1, 3):
        bp = fl.BatchedPlan([5000] * B, None, torch.from_numpy(w).to(dev), 1e-6, shared_nodes=True)
        f = bp.execute(torch.from_numpy(np.tile(c, B)).to(torch.complex64).to(dev)).cpu().numpy()
        bp.close()
        for i in range(B):
            assert np.array_equal(f[i * 700:(i + 1) * 700], ref), (B, i)


def test_per_transform_pointers(fl):
    # one node tensor and one coefficient / result tensor per transform
    # (fl_plan_batched_ptrs, fl_execute_batched_ptrs): the same numbers as
    # the concatenated calls, bit for bit; a transform without nodes included
    Ns = [3000, 700, 12000, 50]
    Ms = [800, 0, 2500, 40]
    cs, ws = _batch(Ns, Ms, seed=90, kinds=("clustered", "disk"))
    dev = torch.device("cuda")
    bp = fl.BatchedPlan(Ns, Ms, [torch.from_numpy(w).to(dev) for w in ws], 1e-6)
    ref_plan = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), 1e-6)
    ct = [torch.from_numpy(c).to(torch.complex64).to(dev) for c in cs]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = bp.execute_list(ct)
        outs2 = bp.execute_list([2 * c for c in ct])     # the pointer table re-read per call
        ref = ref_plan.execute(torch.cat(ct))
    s.synchronize()
    moff = 0
    for i, m in enumerate(Ms):
        assert outs[i].numel() == m
        assert torch.equal(outs[i], ref[moff:moff + m])
        assert torch.allclose(outs2[i], 2 * ref[moff:moff + m], rtol=1e-5, atol=1e-3)
        moff += m
    bp.close()
    ref_plan.close()
