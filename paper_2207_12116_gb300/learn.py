"""Learned branching: data from the solver's own propagation, training on the
library's tensor-core kernels, and the policy as a search strategy.

Data.  Search nodes are random descents of a model's tree (input-order
branching decisions), propagated to their fixed points by pccp_propagate.
At each node with at least two unfixed branch variables every candidate is
probed the way strong branching does: both children of its lower-half split
are propagated (again by pccp_propagate, all children of a batch in one
launch) and scored by the failures they expose and the domain reduction they
cause.  The expert blends this probe with first-fail's preference for small
domains and its tie-break (lower branch index first): a probe alone favours
splits that fail or shrink domains, which makes depth-first dives thrash
before any assignment completes, and without the tie-break the many equal
widths leave the order among tied candidates to noise, which on scheduling
models (tasks numbered in precedence order) loses first-fail's habit of
placing tasks in that order.  The target of a node is the softmax of the
expert's scores over its candidates, and the policy learns to rank
candidates like the expert without running the probe.
Features come from pccp_policy_features, i.e. exactly the values the search
kernels feed the network.

Training.  pccp_policy_train_step: forward, listwise softmax cross-entropy,
backward and Adam, with every matrix product on the tensor cores (BF16
operands, FP32 accumulation).
"""
import numpy as np

from . import Model, Policy, propagate, policy_features, rcpsp
from . import PCCP_FIXPOINT

PROBE_TEMPERATURE = 0.05
WIDTH_WEIGHT = 1.5  # expert score -= WIDTH_WEIGHT * log2(1 + domain width)
INDEX_WEIGHT = 2.0  # expert score -= INDEX_WEIGHT * branch index / branch count


def _device():
    import torch
    return torch.device("cuda", torch.cuda.current_device())


def collect(instances, nodes_per_model=256, seed=0, max_decisions=15, width_weight=WIDTH_WEIGHT,
            index_weight=INDEX_WEIGHT):
    """Training groups from a list of scheduling instances.  Returns a dict of
    CUDA tensors: features [R, 12], group_off [G + 1], target [R].
    width_weight: weight of first-fail's log2(1 + width) in the expert;
    index_weight: weight of its tie-break (lower branch index first)."""
    import torch
    from synthetic import draw_partial_assignments
    dev = _device()
    feats, targets, sizes = [], [], []
    for mi, inst in enumerate(instances):
        rows = rcpsp.build_rows(inst)
        model = Model.from_rows(rows)
        nodes = draw_partial_assignments(inst.n, inst.horizon, nodes_per_model,
                                         seed=seed * 100_003 + mi, max_decisions=max_decisions)
        lb_h, ub_h = rcpsp.node_stores(rows, nodes)
        lb = torch.from_numpy(lb_h).to(dev)
        ub = torch.from_numpy(ub_h).to(dev)
        st, _ = propagate(model, lb, ub)
        ok = (st == PCCP_FIXPOINT).nonzero().flatten()
        if ok.numel() == 0:
            continue
        lb, ub = lb[ok].contiguous(), ub[ok].contiguous()
        depth = torch.tensor([len(nodes[i]) for i in ok.tolist()], dtype=torch.int32, device=dev)
        branch = torch.from_numpy(model.branch.astype(np.int64)).to(dev)
        blb, bub = lb[:, branch], ub[:, branch]
        unfixed = blb < bub                                    # [N, nb]
        keep = unfixed.sum(dim=1) >= 2
        if keep.sum() == 0:
            continue
        lb, ub, depth = lb[keep].contiguous(), ub[keep].contiguous(), depth[keep].contiguous()
        blb, bub, unfixed = blb[keep], bub[keep], unfixed[keep]
        f = policy_features(model, lb, ub, depth)             # [N, nb, 12]
        node_idx, cand = unfixed.nonzero(as_tuple=True)        # candidates
        var = branch[cand]
        mid = blb[node_idx, cand] + (bub[node_idx, cand] - blb[node_idx, cand]) // 2
        # children: left ub(var) <= mid, right lb(var) >= mid + 1
        clb = torch.cat([lb[node_idx], lb[node_idx]]).clone()
        cub = torch.cat([ub[node_idx], ub[node_idx]]).clone()
        c = node_idx.numel()
        ar = torch.arange(c, device=dev)
        cub[ar, var] = torch.minimum(cub[ar, var], mid.to(torch.int32))
        clb[c + ar, var] = torch.maximum(clb[c + ar, var], (mid + 1).to(torch.int32))
        clb, cub = clb.contiguous(), cub.contiguous()
        cst, _ = propagate(model, clb, cub)
        failed = (cst != PCCP_FIXPOINT).float()
        w_before = (bub - blb).float().sum(dim=1)[node_idx].clamp(min=1.0)
        w_after = (cub[:, branch] - clb[:, branch]).float().sum(dim=1)
        red = ((w_before.repeat(2) - w_after) / w_before.repeat(2)) * (1 - failed)
        width = (bub[node_idx, cand] - blb[node_idx, cand]).float()
        score = (failed[:c] + failed[c:]) * 2.0 + red[:c] + red[c:] \
            - width_weight * torch.log2(1.0 + width) \
            - index_weight * cand.float() / float(branch.numel())
        # groups: one per node, candidates in row-major order of (node, branch index)
        counts = torch.bincount(node_idx, minlength=lb.shape[0])
        target = torch.empty_like(score)
        off = 0
        for cnt in counts.tolist():
            s = score[off:off + cnt] / PROBE_TEMPERATURE
            target[off:off + cnt] = torch.softmax(s, dim=0)
            off += cnt
        feats.append(f[node_idx, cand])
        targets.append(target)
        sizes.append(counts[counts > 0])
    features = torch.cat(feats).contiguous()
    target = torch.cat(targets).contiguous()
    sizes = torch.cat(sizes)
    group_off = torch.zeros(sizes.numel() + 1, dtype=torch.int32, device=dev)
    group_off[1:] = torch.cumsum(sizes, 0).to(torch.int32)
    return {"features": features, "group_off": group_off, "target": target}


def batches(data, groups_per_batch, seed):
    """Random mini-batches of whole groups (features, group_off, target)."""
    import torch
    g = np.random.default_rng(seed)
    off = data["group_off"].cpu().numpy()
    n_groups = off.size - 1
    order = g.permutation(n_groups)
    for b in range(0, n_groups, groups_per_batch):
        sel = np.sort(order[b:b + groups_per_batch])
        idx = np.concatenate([np.arange(off[i], off[i + 1]) for i in sel])
        sizes = off[sel + 1] - off[sel]
        go = np.zeros(sel.size + 1, dtype=np.int32)
        go[1:] = np.cumsum(sizes)
        it = torch.from_numpy(idx).to(data["features"].device)
        yield (data["features"][it].contiguous(), torch.from_numpy(go).to(it.device),
               data["target"][it].contiguous())


def train(policy: Policy, data, epochs=4, groups_per_batch=256, lr=2e-3, seed=0):
    """Adam epochs over the data; returns the mean loss of every epoch."""
    losses = []
    for e in range(epochs):
        ls = [policy.train_step(f, go, t, lr=lr) for f, go, t in
              batches(data, groups_per_batch, seed + e)]
        losses.append(float(np.mean(ls)))
    return losses


def ranking_accuracy(policy: Policy, data):
    """Fraction of groups whose highest-scoring candidate is the target's."""
    s = policy.score(data["features"]).cpu().numpy()
    t = data["target"].cpu().numpy()
    off = data["group_off"].cpu().numpy()
    hits = [int(np.argmax(s[a:b]) == np.argmax(t[a:b])) for a, b in zip(off[:-1], off[1:])]
    return float(np.mean(hits))


ROLLOUT_TEMPERATURE = 0.35  # target = softmax(-log2(1 + proof nodes) / T)


def collect_rollouts(instances, nodes_per_model=24, seed=0, node_cap=20000,
                     temperature=ROLLOUT_TEMPERATURE, mode="soft", record=None):
    """Training groups whose targets come from measured proof trees.

    For each instance: its optimum z (a parallel search); then search nodes
    of the proof phase, i.e. with ub(objective) <= z - 1, reached by descents
    that split first-fail's variable on a random side and are propagated by
    pccp_propagate level by level.  At each node with at least two unfixed
    branch variables every candidate v is scored by the size of the two
    first-fail proof trees below its lower-half split: each child becomes a
    model whose root box is the child's store, and all children of all nodes
    are proved infeasible in one parallel batch (pccp_solve_batch over a
    shared queue, node_cap nodes per child at most).  The target of a node is
    softmax(-log2(1 + nodes(v)) / temperature) over its candidates (or
    another form, see rollout_targets): one step of policy improvement over
    first-fail, learned without running a single rollout at search time.
    Returns (data, stats) with data as collect() plus the raw proof sizes
    ("cost") and domain widths ("width") of the candidates.  record: a list
    that receives (instance, child lb0, child ub0, nodes, status) for every
    child proved."""
    import torch
    from . import solve, solve_batch, PCCP_FIRST_FAIL, PCCP_RES_LIMIT
    dev = _device()
    g = np.random.default_rng(seed)
    feats, targets, sizes, widths = [], [], [], []
    n_children = n_capped = 0
    for inst in instances:
        rows = rcpsp.build_rows(inst)
        model = Model.from_rows(rows)
        z = solve(model, strategy=PCCP_FIRST_FAIL, deterministic=False)["objective"]
        M = int(rows["objective"])
        branch = np.asarray(rows["branch"], dtype=np.int64)
        base_lb, base_ub = rows["lb0"].copy(), rows["ub0"].copy()
        base_ub[M] = z - 1  # the proof phase: nothing better than z exists
        # descents: first-fail's variable, random side, until failure or
        # every branch variable is fixed; every visited node is a candidate
        K = nodes_per_model
        lb = np.tile(base_lb, (K, 1))
        ub = np.tile(base_ub, (K, 1))
        alive = np.ones(K, dtype=bool)
        pool = []  # (lb, ub, depth)
        for depth in range(64):
            idx = np.nonzero(alive)[0]
            if idx.size == 0:
                break
            dlb = torch.from_numpy(lb[idx]).to(dev)
            dub = torch.from_numpy(ub[idx]).to(dev)
            st, _ = propagate(model, dlb, dub)
            st = st.cpu().numpy()
            plb, pub = dlb.cpu().numpy(), dub.cpu().numpy()
            for r, i in enumerate(idx):
                if st[r] != PCCP_FIXPOINT:
                    alive[i] = False
                    continue
                w = pub[r, branch] - plb[r, branch]
                open_ = np.nonzero(w > 0)[0]
                if open_.size >= 2:
                    pool.append((plb[r].copy(), pub[r].copy(), depth))
                if open_.size == 0:
                    alive[i] = False
                    continue
                k = open_[np.argmin(w[open_])]  # first-fail, ties to the lower index
                v = branch[k]
                m = plb[r, v] + (pub[r, v] - plb[r, v]) // 2
                lb[i], ub[i] = plb[r], pub[r]
                if g.random() < 0.5:
                    ub[i, v] = m
                else:
                    lb[i, v] = m + 1
        if not pool:
            continue
        pick = g.choice(len(pool), size=min(nodes_per_model, len(pool)), replace=False)
        nodes = [pool[p] for p in sorted(pick)]
        child_models, owner = [], []
        for ni, (nlb, nub, depth) in enumerate(nodes):
            for k in np.nonzero(nub[branch] > nlb[branch])[0]:
                v = branch[k]
                m = nlb[v] + (nub[v] - nlb[v]) // 2
                for side in (0, 1):
                    clb, cub = nlb.copy(), nub.copy()
                    if side == 0:
                        cub[v] = m
                    else:
                        clb[v] = m + 1
                    crow = dict(rows)
                    crow["lb0"], crow["ub0"] = clb, cub
                    child_models.append(Model.from_rows(crow))
                    owner.append((ni, int(k)))
        res = solve_batch(child_models, strategy=PCCP_FIRST_FAIL, deterministic=False,
                          node_limit=node_cap)
        n_children += len(res)
        n_capped += sum(r["status"] == PCCP_RES_LIMIT for r in res)
        cost = {}
        for ci, ((ni, k), r) in enumerate(zip(owner, res)):
            cost[(ni, k)] = cost.get((ni, k), 0) + r["nodes"]
            if record is not None:  # (instance, child root box, nodes, status)
                record.append((inst, child_models[ci].lb0.copy(), child_models[ci].ub0.copy(),
                               r["nodes"], r["status"]))
        for cm in child_models:
            cm.close()
        nlb_t = torch.from_numpy(np.stack([n[0] for n in nodes])).to(dev)
        nub_t = torch.from_numpy(np.stack([n[1] for n in nodes])).to(dev)
        dep_t = torch.tensor([n[2] for n in nodes], dtype=torch.int32, device=dev)
        f = policy_features(model, nlb_t, nub_t, dep_t)  # [N, nb, 12]
        for ni in range(len(nodes)):
            ks = sorted(k for (n2, k) in cost if n2 == ni)
            nlb, nub = nodes[ni][0], nodes[ni][1]
            feats.append(f[ni, ks])
            targets.append(torch.tensor([cost[(ni, k)] for k in ks], dtype=torch.float32,
                                        device=dev))
            widths.append(torch.tensor([nub[branch[k]] - nlb[branch[k]] for k in ks],
                                       dtype=torch.float32, device=dev))
            sizes.append(len(ks))
        model.close()
    features = torch.cat(feats).contiguous()
    cost = torch.cat(targets).contiguous()
    group_off = torch.zeros(len(sizes) + 1, dtype=torch.int32, device=dev)
    group_off[1:] = torch.cumsum(torch.tensor(sizes, device=dev), 0).to(torch.int32)
    data = {"features": features, "group_off": group_off, "cost": cost,
            "width": torch.cat(widths).contiguous()}
    rollout_targets(data, mode, temperature)
    return data, {"groups": len(sizes), "children": n_children, "children_capped": n_capped}


def rollout_targets(data, mode="soft", temperature=ROLLOUT_TEMPERATURE, width_weight=1.0):
    """Targets from the measured proof sizes of collect_rollouts, per group:
      soft    softmax(-log2(1 + nodes) / temperature);
      hard    all mass on the smallest proof, ties to first-fail's choice
              (smallest width, then the lower index);
      soft_ff softmax(-(log2(1 + nodes) + width_weight * log2(1 + width)) / T):
              the proof sizes with first-fail's preference as a prior."""
    import torch
    off = data["group_off"].cpu().numpy()
    c = torch.log2(1.0 + data["cost"])
    w = torch.log2(1.0 + data["width"])
    t = torch.empty_like(c)
    for a, b in zip(off[:-1], off[1:]):
        if mode == "hard":
            cc, ww = data["cost"][a:b].cpu().numpy(), data["width"][a:b].cpu().numpy()
            best = min(range(b - a), key=lambda i: (cc[i], ww[i], i))
            t[a:b] = 0.0
            t[a + best] = 1.0
        elif mode == "soft_ff":
            t[a:b] = torch.softmax(-(c[a:b] + width_weight * w[a:b]) / temperature, dim=0)
        else:
            t[a:b] = torch.softmax(-c[a:b] / temperature, dim=0)
    data["target"] = t.contiguous()
    return data
