"""Learned branching on the GPU: the tensor-core MLP against a plain PyTorch
FP32 reference (with the same BF16 roundings), the feature kernel against a
NumPy restatement, the training step against PyTorch autograd, and the
learned strategy inside complete searches (optima unchanged)."""
import numpy as np
import pytest

import oracle
from oracle import brute
from oracle.rcpsp import rcpsp_model
import paper_2207_12116_gb300 as pccp
from paper_2207_12116_gb300 import learn
from synthetic import config_instance, draw_partial_assignments

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def bf(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float32)


def ref_scores(w, x):
    """Plain PyTorch FP32 forward with the network's BF16 roundings: inputs,
    weights of layers 1-2 and the first hidden layer are BF16."""
    xb = bf(x)
    h1 = torch.relu(xb @ bf(w["w1"]).T + torch.tensor(w["b1"]))
    h2 = torch.relu(bf(h1) @ bf(w["w2"]).T + torch.tensor(w["b2"]))
    return h2 @ torch.tensor(w["w3"]) + w["b3"]


def test_scores_match_pytorch_reference():
    g = np.random.default_rng(3)
    for seed in range(3):
        pol = pccp.Policy.random(seed)
        w = pol.weights()
        x = g.uniform(-1, 2, (333, 12)).astype(np.float32)
        s = pol.score(torch.from_numpy(x).cuda()).cpu()
        r = ref_scores(w, x)
        tol = 1e-2 * float(r.abs().max()) + 1e-3
        assert torch.allclose(s, r, atol=tol, rtol=1e-2), float((s - r).abs().max())


def test_features_match_numpy_restatement():
    """Every feature against its definition on the scheduling instance
    itself (degrees, offsets, demand = sum over resources of usage /
    capacity), not on the packed rows."""
    inst = config_instance("j30", 2)
    rows = pccp.rcpsp.build_rows(inst)
    m = pccp.Model.from_rows(rows)
    nodes = draw_partial_assignments(inst.n, inst.horizon, 40, seed=8)
    lb, ub = pccp.rcpsp.node_stores(rows, nodes)
    depth = np.array([len(d) for d in nodes], dtype=np.int32)
    f = pccp.policy_features(m, torch.from_numpy(lb).cuda(), torch.from_numpy(ub).cuda(),
                             torch.from_numpy(depth).cuda()).cpu().numpy()
    n, M = inst.n, inst.n + inst.n * inst.n
    out_deg = np.zeros(n)
    sum_d = np.zeros(n)
    in_deg = np.zeros(n)
    for (x, y, d) in rows["temporal"]:
        if x < n:
            out_deg[x] += 1
            sum_d[x] += d
        if y < n:
            in_deg[y] += 1
    n_rf = np.zeros(n)
    for (b, x, y, d) in rows["reified"]:
        n_rf[x] += 1
        n_rf[y] += 1
    # demand of task k: its usages over the capacities, summed over resources
    demand = np.array([sum(inst.usage[r][k] / inst.capacity[r] for r in range(inst.n_resources))
                       for k in range(n)])
    lb0, ub0 = rows["lb0"], rows["ub0"]
    for s in range(len(nodes)):
        for k in range(n):
            w0 = ub0[k] - lb0[k]
            inv = np.float32(1.0) / np.float32(w0 + 1)
            l, u = max(lb[s, k], lb0[k]), min(ub[s, k], ub0[k])
            prog = np.float32(max(lb[s, M], lb0[M]) - lb0[M]) / np.float32(ub0[M] - lb0[M] + 1)
            ref = [np.float32(l - lb0[k]) * inv, np.float32(u - lb0[k]) * inv,
                   np.float32(u - l) * inv, np.log2(np.float32(1 + u - l)) / 16,
                   out_deg[k] / 8, sum_d[k] * inv, in_deg[k] / 8, n_rf[k] / 64,
                   demand[k] / 4,
                   k / n, depth[s] / (depth[s] + 32.0), prog]
            refb = bf(np.array(ref, dtype=np.float32)).numpy()
            assert np.allclose(f[s, k], refb, rtol=2 ** -7, atol=1e-6), (s, k, f[s, k], refb)


def _random_groups(seed, n_groups=48):
    g = np.random.default_rng(seed)
    sizes = g.integers(2, 9, n_groups)
    off = np.zeros(n_groups + 1, dtype=np.int32)
    off[1:] = np.cumsum(sizes)
    x = g.uniform(0, 1, (off[-1], 12)).astype(np.float32)
    t = np.zeros(off[-1], dtype=np.float32)
    for i in range(n_groups):  # target: the candidate with the largest feature 2
        t[off[i] + np.argmax(x[off[i]:off[i + 1], 2])] = 1.0
    return x, off, t


def test_first_training_step_follows_autograd():
    """The gradient of the mean listwise cross-entropy equals PyTorch
    autograd's on the same BF16-rounded forward (rounding passed straight
    through), element by element; and Adam's first step moves each weight by
    about -lr * sign(gradient)."""
    pol = pccp.Policy.random(11)
    w0 = pol.weights()
    x, off, t = _random_groups(5)
    lr = 1e-3
    loss = pol.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda(),
                          torch.from_numpy(t).cuda(), lr=lr)
    w1 = pol.weights()
    P = {k: torch.tensor(w0[k], requires_grad=True) for k in ("w1", "b1", "w2", "b2", "w3")}
    b3 = torch.tensor(w0["b3"], requires_grad=True)
    ste = lambda a: a + (bf(a.detach()) - a).detach()  # BF16 value, identity gradient
    h1 = torch.relu(ste(torch.from_numpy(x)) @ ste(P["w1"]).T + P["b1"])
    h2 = torch.relu(ste(h1) @ ste(P["w2"]).T + P["b2"])
    s = h2 @ P["w3"] + b3
    tt = torch.from_numpy(t)
    L = 0
    for i in range(len(off) - 1):
        a, b = off[i], off[i + 1]
        L = L - (tt[a:b] * torch.log_softmax(s[a:b], 0)).sum()
    L = L / (len(off) - 1)
    L.backward()
    assert abs(loss - L.item()) < 1e-2 * max(1.0, abs(L.item()))
    # the raw gradient, element by element: the kernels feed BF16 copies of
    # the activations and of dZ into the tensor-core GEMMs (FP32 accumulate),
    # so each entry may differ by a few BF16 roundings of the largest terms
    got = pol.gradients()
    for k in ("w1", "b1", "w2", "b2", "w3"):
        gr = P[k].grad.numpy()
        tol = 2e-2 * np.abs(gr).max() + 1e-6
        err = np.abs(got[k] - gr)
        assert err.max() <= tol, (k, float(err.max()), float(tol))
        assert np.corrcoef(got[k].ravel(), gr.ravel())[0, 1] > 0.999, k
    assert abs(got["b3"] - float(b3.grad)) <= 2e-2 * abs(float(b3.grad)) + 1e-6
    for k in ("w1", "b1", "w2", "b2", "w3"):
        gr = P[k].grad.numpy()
        upd = w1[k] - w0[k]
        big = np.abs(gr) > 0.05 * np.abs(gr).max()
        assert big.sum() > 0
        agree = np.mean(np.sign(upd[big]) == -np.sign(gr[big]))
        assert agree > 0.97, (k, agree)
        assert np.allclose(np.abs(upd[big]), lr, rtol=0.05)


def test_training_learns_a_ranking():
    pol = pccp.Policy.random(12)
    x, off, t = _random_groups(6, n_groups=512)
    data = {"features": torch.from_numpy(x).cuda(), "group_off": torch.from_numpy(off).cuda(),
            "target": torch.from_numpy(t).cuda()}
    before = learn.ranking_accuracy(pol, data)
    losses = learn.train(pol, data, epochs=30, groups_per_batch=128, lr=3e-3)
    after = learn.ranking_accuracy(pol, data)
    assert losses[-1] < 0.5 * losses[0]
    assert after > 0.9 and after > before


@pytest.mark.parametrize("deterministic", [True, False])
def test_learned_search_keeps_optima(deterministic):
    pol = pccp.Policy.random(21)
    for seed in range(0, 100, 9):
        inst = config_instance("tiny8", seed)
        m = pccp.Model.from_rcpsp(inst)
        r = pccp.solve(m, strategy=pccp.PCCP_LEARNED, policy=pol, deterministic=deterministic)
        o = oracle.solve(rcpsp_model(inst))
        assert r["status"] == pccp.PCCP_RES_OPTIMAL and r["objective"] == o["objective"]
        s = [int(v) for v in r["witness"][:inst.n]]
        assert brute.rcpsp_feasible(inst, s)
        if deterministic:  # the deterministic walk is reproducible
            r2 = pccp.solve(m, strategy=pccp.PCCP_LEARNED, policy=pol)
            assert (r2["nodes"], r2["fails"], r2["solutions"]) == (r["nodes"], r["fails"], r["solutions"])


def test_learned_batched_and_count_all():
    pol = pccp.Policy.random(22)
    insts = [config_instance("tiny8", s) for s in range(20)]
    res = pccp.solve_batch([pccp.Model.from_rcpsp(i) for i in insts], strategy=pccp.PCCP_LEARNED,
                           policy=pol)
    for inst, r in zip(insts, res):
        om = rcpsp_model(inst)
        o = oracle.solve(om)
        assert r["objective"] == o["objective"]
        # every order visits the same solutions: count-all agrees
        c = oracle.solve(om, mode=oracle.COUNT_ALL, obj_ub=o["objective"])
        rc = pccp.solve(pccp.Model.from_rcpsp(inst), mode=pccp.PCCP_COUNT_ALL,
                        obj_ub=o["objective"], strategy=pccp.PCCP_LEARNED, policy=pol)
        assert rc["solutions"] == c["solutions"]


def test_pipeline_collects_and_trains():
    insts = [config_instance("tiny8", s) for s in range(6)] + \
            [config_instance("j30", s) for s in range(2)]
    data = learn.collect(insts, nodes_per_model=128, seed=1)
    n_groups = data["group_off"].numel() - 1
    assert n_groups > 100
    off = data["group_off"].cpu().numpy()
    t = data["target"].cpu().numpy()
    assert np.allclose([t[a:b].sum() for a, b in zip(off[:-1], off[1:])], 1.0, atol=1e-4)
    pol = pccp.Policy.random(5)
    # the loss cannot fall below the targets' entropy; what is learnable is the
    # divergence above it and the top-1 agreement with the probe
    ent = -float(np.mean([np.sum(t[a:b] * np.log(np.maximum(t[a:b], 1e-30)))
                          for a, b in zip(off[:-1], off[1:])]))
    acc0 = learn.ranking_accuracy(pol, data)
    losses = learn.train(pol, data, epochs=10, groups_per_batch=128, lr=2e-3)
    acc1 = learn.ranking_accuracy(pol, data)
    assert losses[-1] - ent < 0.8 * (losses[0] - ent)
    assert acc1 > acc0


def test_rollout_labels_are_oracle_proof_sizes():
    """The rollout labels of learn.collect_rollouts: every child subproblem's
    node count is the size of its first-fail proof tree (objective bounded
    below the optimum, so no solution and an order-free count), equal to the
    oracle's on the same child box; targets are distributions over each
    node's candidates."""
    insts = [config_instance("mixed6_10", 5000 + s) for s in range(4)]
    rec = []
    data, stats = learn.collect_rollouts(insts, nodes_per_model=3, seed=2, node_cap=10 ** 8,
                                         record=rec)
    assert stats["groups"] > 0 and stats["children_capped"] == 0 and len(rec) == stats["children"]
    off = data["group_off"].cpu().numpy()
    t = data["target"].cpu().numpy()
    for a, b in zip(off[:-1], off[1:]):
        assert b - a >= 2 and abs(t[a:b].sum() - 1) < 1e-4
    small = [r for r in rec if r[3] <= 20000][:60]  # the oracle re-proves these on the CPU
    assert len(small) >= 20
    for inst, lb0, ub0, nodes, status in small:
        om = rcpsp_model(inst)
        child = oracle.Model(lb0, ub0, om.temporal, om.linear, om.reified, om.objective, om.branch)
        o = oracle.solve(child, strategy=oracle.FIRST_FAIL)
        assert o["status"] == oracle.RES_INFEASIBLE
        assert nodes == o["nodes"] and status == pccp.PCCP_RES_INFEASIBLE
