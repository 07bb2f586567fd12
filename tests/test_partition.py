"""Partition and halo plans (mfd_partition_*, mfd_halo_*): host-only index
structures for running the leapfrog of Eq. 19 with the nodes split over
several GPUs. No GPU is used: the plans are checked for their invariants, and
a sharded leapfrog over them (numpy stencil sums on each shard, one halo
exchange after each half step) reproduces the oracle's whole-domain run, both
with every shard in one process and with two gloo ranks."""
import socket

import numpy as np
import pytest

import oracle as O
import workloads as W

M = pytest.importorskip("paper_2508_18205_gb300")

S_C, C_HV = 0.5, 4e-3


def morton_order(xyz, bits=10):
    """Caller ids sorted along a Morton curve of the bounding box (a test-side
    ordering; the partition takes any permutation)."""
    lo, hi = xyz.min(0), xyz.max(0)
    q = np.minimum(((xyz - lo) / np.maximum(hi - lo, 1e-300) * (2 ** bits)).astype(np.int64), 2 ** bits - 1)
    key = np.zeros(len(xyz), dtype=np.int64)
    for b in range(bits):
        for a in range(xyz.shape[1]):
            key |= ((q[:, a] >> b) & 1) << (b * xyz.shape[1] + a)
    return np.argsort(key, kind="stable")


# ------------------------------------------------------------- plan invariants

def test_ranges_cover_the_set_with_balanced_sizes():
    n = 1001
    order = np.random.default_rng(1).permutation(n)
    for S in (1, 2, 3, 7, 64):
        p = M.Partition(n, S, order)
        owner = p.owner()
        sizes = [len(p.owned(s)) for s in range(S)]
        assert sum(sizes) == n and max(sizes) - min(sizes) <= 1
        allown = np.concatenate([p.owned(s) for s in range(S)])
        assert np.array_equal(allown, order)  # contiguous ranges of the order
        for s in range(S):
            assert np.all(owner[p.owned(s)] == s)


def test_more_shards_than_nodes_gives_empty_shards():
    p = M.Partition(3, 5)
    assert sorted(len(p.owned(s)) for s in range(5)) == [0, 0, 1, 1, 1]
    idx = np.array([[0, 1], [1, 2], [2, 0]])
    h = M.HaloPlan(p, [(p, idx)])
    for s in range(5):
        assert h.local_idx(s, 0).shape == (len(p.owned(s)), 2)


def _staggered_idx(nx=24, seed=3):
    e = W.periodic_box((nx, nx), 0.25, seed)
    h = W.periodic_box((nx, nx), 0.25, seed + 1, offset=(0.5, 0.5))
    per = e.period
    return e, h, {"he": O.knn(h.xyz, e.xyz, per, 30), "hh": O.knn(h.xyz, h.xyz, per, 57),
                  "eh": O.knn(e.xyz, h.xyz, per, 30), "ee": O.knn(e.xyz, e.xyz, per, 57)}


@pytest.mark.parametrize("S", [1, 2, 5])
def test_halo_plan_invariants(S):
    e, h, I = _staggered_idx()
    pe = M.Partition(e.n, S, morton_order(e.xyz))
    ph = M.Partition(h.n, S, morton_order(h.xyz))
    plan_e = M.HaloPlan(pe, [(ph, I["he"]), (pe, I["ee"])])  # sources: the E set
    plan_h = M.HaloPlan(ph, [(pe, I["eh"]), (ph, I["hh"])])  # sources: the H set
    for plan, src, sets in ((plan_e, pe, [(ph, I["he"]), (pe, I["ee"])]),
                            (plan_h, ph, [(pe, I["eh"]), (ph, I["hh"])])):
        owner = src.owner()
        for s in range(S):
            own, halo = src.owned(s), plan.nodes(s)
            assert len(np.intersect1d(own, halo)) == 0
            assert np.all(owner[halo] != s)
            # ordered by owner, then by position in the partition order
            pos = np.empty(src.n, dtype=np.int64)
            pos[np.concatenate([src.owned(q) for q in range(S)])] = np.arange(src.n)
            assert np.all(np.diff(pos[halo]) > 0)
            # the receiver's halo is the concatenation of what every shard sends it
            sent = [plan.send(q, s) for q in range(S)]
            assert len(sent[s]) == 0
            assert np.array_equal(np.concatenate(sent), halo)
            local = np.concatenate([own, halo])
            used = np.zeros(len(local), dtype=bool)
            for k, (cp, idx) in enumerate(sets):
                L = plan.local_idx(s, k)
                rows = cp.owned(s)
                assert L.min(initial=0) >= 0 and L.max(initial=-1) < len(local)
                # localised stencils read exactly the original neighbours, in order
                assert np.array_equal(local[L], idx[rows])
                used[L.reshape(-1)] = True
            # the halo is minimal: every halo node is read by an owned stencil
            assert used[len(own):].all()
        if S == 1:
            assert len(plan.nodes(0)) == 0


def test_halo_shrinks_relative_to_shard_with_morton_order():
    """With the Morton order the halo of a shard scales like its boundary: on a
    periodic 96 x 96 set in 4 quadrant-like shards of 48 x 48 it is about four
    sides of three node rows (stencil radius ~3 h), far below what a random
    order gives."""
    e = W.periodic_box((96, 96), 0.25, 9)
    idx = O.knn(e.xyz, e.xyz, e.period, 31)
    p = M.Partition(e.n, 4, morton_order(e.xyz))
    plan = M.HaloPlan(p, [(p, idx)])
    frac = max(len(plan.nodes(s)) / len(p.owned(s)) for s in range(4))
    assert frac < 0.3, frac
    rnd = M.Partition(e.n, 4, np.random.default_rng(0).permutation(e.n))
    plan_r = M.HaloPlan(rnd, [(rnd, idx)])
    assert min(len(plan_r.nodes(s)) for s in range(4)) > 2 * max(len(plan.nodes(s)) for s in range(4))


def test_bad_arguments_raise():
    with pytest.raises(M.MfdError):
        M.Partition(4, 0)
    with pytest.raises(M.MfdError):
        M.Partition(4, 2, [0, 1, 1, 3])
    p = M.Partition(4, 2)
    with pytest.raises(M.MfdError):
        M.HaloPlan(p, [(p, np.array([[0, 4], [1, 2], [2, 3], [3, 0]]))])
    q = M.Partition(4, 3)
    with pytest.raises(M.MfdError):
        M.HaloPlan(p, [(q, np.zeros((4, 2), dtype=np.int64))])
    with pytest.raises(M.MfdError):
        p.owned(2)


# ------------------------------------------------------- sharded leapfrog

class ShardedTMz:
    """The TMz leapfrog of Eq. 19 run shard by shard over the halo plans.

    Shard s keeps, per field, one array [owned values | halo values]; its
    stencils are the plans' localised indices, its weights the oracle's rows
    of the centres it owns. After the H half step every shard sends the H
    values its neighbours' halos hold, after the E half step the E values."""

    def __init__(self, prob, e_nodes, h_nodes, S, sources=None):
        self.p, self.S = prob, S
        pe = M.Partition(prob.ne, S, morton_order(e_nodes.xyz))
        ph = pe if h_nodes is e_nodes else M.Partition(prob.nh, S, morton_order(h_nodes.xyz))
        plan_e = M.HaloPlan(pe, [(ph, prob.hc.idx), (pe, prob.ev.idx)])  # reads of the E set
        plan_h = M.HaloPlan(ph, [(pe, prob.ec.idx), (ph, prob.hv.idx)])  # reads of the H set
        self.sh = []
        for s in range(S):
            oe, oh = pe.owned(s), ph.owned(s)
            d = dict(oe=oe, oh=oh, he=plan_e.nodes(s), hh=plan_h.nodes(s),
                     hc_l=plan_e.local_idx(s, 0), hc_w=prob.hc.w[:, oh, :],
                     hv_l=plan_h.local_idx(s, 1), hv_w=prob.hv.w[0, oh, :],
                     ec_l=plan_h.local_idx(s, 0), ec_w=prob.ec.w[:, oe, :],
                     ev_l=plan_e.local_idx(s, 1), ev_w=prob.ev.w[0, oe, :],
                     ce=prob.dt / (prob.eps0 * prob.eps_r[oe]), pec=prob.pec[oe].astype(bool))
            inv_e = np.full(prob.ne, -1)
            inv_e[oe] = np.arange(len(oe))
            inv_h = np.full(prob.nh, -1)
            inv_h[oh] = np.arange(len(oh))
            # what s sends to q, as positions among s's owned values
            d["send_e"] = {q: inv_e[plan_e.send(s, q)] for q in range(S) if q != s}
            d["send_h"] = {q: inv_h[plan_h.send(s, q)] for q in range(S) if q != s}
            d["recv_e"] = {q: len(plan_e.send(q, s)) for q in range(S) if q != s}
            d["recv_h"] = {q: len(plan_h.send(q, s)) for q in range(S) if q != s}
            if sources is not None:
                mine = inv_e[sources.node] >= 0
                d["src"] = (inv_e[sources.node[mine]], sources.amp[mine], sources.f0[mine], sources.t0[mine])
            else:
                d["src"] = None
            self.sh.append(d)

    def h_pass(self, s, ez, hx, hy):
        d, p = self.sh[s], self.p
        ch = p.dt / p.mu0
        dxE = np.sum(d["hc_w"][0] * ez[d["hc_l"]], axis=1)
        dyE = np.sum(d["hc_w"][1] * ez[d["hc_l"]], axis=1)
        vx = np.sum(d["hv_w"] * hx[d["hv_l"]], axis=1)
        vy = np.sum(d["hv_w"] * hy[d["hv_l"]], axis=1)
        m = len(d["oh"])
        return hx[:m] - ch * (dyE - p.gamma * vx), hy[:m] + ch * (dxE + p.gamma * vy)

    def e_pass(self, s, step, ez, hx1, hy1):
        d, p = self.sh[s], self.p
        dxH = np.sum(d["ec_w"][0] * hy1[d["ec_l"]], axis=1)
        dyH = np.sum(d["ec_w"][1] * hx1[d["ec_l"]], axis=1)
        ve = np.sum(d["ev_w"] * ez[d["ev_l"]], axis=1)
        m = len(d["oe"])
        ez1 = ez[:m] + d["ce"] * (dxH - dyH + p.gamma * ve)
        if d["src"] is not None:
            t1 = (step + 1) * p.dt
            for i, a, f, t0 in zip(*d["src"]):
                ez1[i] += a * O.ricker(t1, f, t0)
        ez1[d["pec"]] = 0.0
        return ez1


def _problem(kind):
    dt, eps0, mu0, c0, eta0 = W.units(S_C)
    if kind == "staggered":
        e = W.periodic_box((20, 20), 0.25, 11)
        h = W.periodic_box((20, 20), 0.25, 12, offset=(0.5, 0.5))
        prob = O.tmz_staggered(e, h, 30, 5, 4, 3, dt, eps0, mu0, 4e-5)
        return prob, e, h, None
    e = W.pec_box((21, 17), 0.25, 13)
    prob, _ = O.tmz_collocated(e, 12, 3, 2, 2, dt, eps0, mu0, -C_HV,
                               eps_r=1.0 + 0.5 * np.random.default_rng(2).random(e.n))
    return prob, e, e, W.ricker_sources(e, 3, 14, c0)


def _initial(prob):
    rng = np.random.default_rng(7)
    return rng.standard_normal(prob.ne), rng.standard_normal(prob.nh), rng.standard_normal(prob.nh)


NSTEPS = 30


@pytest.mark.parametrize("kind", ["staggered", "collocated"])
@pytest.mark.parametrize("S", [3, 4])
def test_sharded_leapfrog_matches_whole_domain_oracle(kind, S):
    prob, e, h, src = _problem(kind)
    ez0, hx0, hy0 = _initial(prob)
    T = ShardedTMz(prob, e, h, S, src)
    ez = [ez0[d["oe"]] for d in T.sh]
    hx = [hx0[d["oh"]] for d in T.sh]
    hy = [hy0[d["oh"]] for d in T.sh]

    def with_halo(vals, s, key):
        d = T.sh[s]
        parts = [vals[s]]
        for q in range(S):
            if q != s:
                parts.append(vals[q][T.sh[q]["send_" + key][s]])
        return np.concatenate(parts)

    for step in range(NSTEPS):
        ezl = [with_halo(ez, s, "e") for s in range(S)]
        hxl = [with_halo(hx, s, "h") for s in range(S)]
        hyl = [with_halo(hy, s, "h") for s in range(S)]
        new_h = [T.h_pass(s, ezl[s], hxl[s], hyl[s]) for s in range(S)]
        hx = [a for a, _ in new_h]
        hy = [b for _, b in new_h]
        hxl = [with_halo(hx, s, "h") for s in range(S)]
        hyl = [with_halo(hy, s, "h") for s in range(S)]
        ez = [T.e_pass(s, step, ezl[s], hxl[s], hyl[s]) for s in range(S)]
    got_e, got_x, got_y = np.zeros(prob.ne), np.zeros(prob.nh), np.zeros(prob.nh)
    for s, d in enumerate(T.sh):
        got_e[d["oe"]], got_x[d["oh"]], got_y[d["oh"]] = ez[s], hx[s], hy[s]
    ref = O.run_tmz(prob, ez0, hx0, hy0, NSTEPS, sources=src)
    got = np.concatenate([got_e, got_x, got_y])
    want = np.concatenate(ref[:3])
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gloo_rank(rank, world, port, kind, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        prob, e, h, src = _problem(kind)
        ez0, hx0, hy0 = _initial(prob)
        T = ShardedTMz(prob, e, h, world, src)
        d = T.sh[rank]

        def exchange(vals, key):
            """Own values -> [own | halo] through point-to-point gloo messages
            (halo blocks arrive in ascending sender order)."""
            reqs, bufs = [], {}
            for peer in range(world):
                if peer == rank:
                    continue
                out = d["send_" + key][peer]
                if len(out):
                    reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(vals[..., out])), peer))
                cnt = d["recv_" + key][peer]
                if cnt:
                    bufs[peer] = torch.empty(vals.shape[:-1] + (cnt,), dtype=torch.float64)
                    reqs.append(dist.irecv(bufs[peer], peer))
            for r in reqs:
                r.wait()
            return np.concatenate([vals] + [bufs[p].numpy() for p in sorted(bufs)], axis=-1)

        ez, hx, hy = ez0[d["oe"]], hx0[d["oh"]], hy0[d["oh"]]
        for step in range(NSTEPS):
            ezl = exchange(ez, "e")
            hl = exchange(np.stack([hx, hy]), "h")
            hx, hy = T.h_pass(rank, ezl, hl[0], hl[1])
            hl = exchange(np.stack([hx, hy]), "h")
            ez = T.e_pass(rank, step, ezl, hl[0], hl[1])
        q.put((rank, d["oe"], d["oh"], ez, hx, hy))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["staggered", "collocated"])
def test_two_gloo_ranks_step_their_shards(kind):
    """World size 2 on CPU: each rank steps only the nodes it owns and learns
    its halo by point-to-point messages; the assembled result equals the
    oracle's whole-domain run."""
    import multiprocessing as mp
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, kind, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    prob, e, h, src = _problem(kind)
    ez0, hx0, hy0 = _initial(prob)
    got_e, got_x, got_y = np.zeros(prob.ne), np.zeros(prob.nh), np.zeros(prob.nh)
    for rank, oe, oh, ez, hx, hy in res:
        got_e[oe], got_x[oh], got_y[oh] = ez, hx, hy
    ref = O.run_tmz(prob, ez0, hx0, hy0, NSTEPS, sources=src)
    got = np.concatenate([got_e, got_x, got_y])
    want = np.concatenate(ref[:3])
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
