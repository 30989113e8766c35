"""Sharding one instance's plate over processes: the host-side split, the sum
of the root's plate sums over a world-size-2 gloo group, and the result
against the single-process oracle.

On the CPU the per-shard compute is the FP64 oracle (``OracleEngine`` below,
test infrastructure): ``shard_forward`` sums its children's log mean-exp
tables into G_r; ``shard_finish`` re-runs the shard's sub-model with the other
shards' share of G added to the root (the oracle's ``root_extra``).  The
product code under test is ``paper_2503_08264_gb300.shard``: the ranges, the
sub-models and their parent remapping, the all-reduce, the reassembly.  The
same split runs through the CUDA entry points in ``test_shard_gpu.py``.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import chain as OC  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2503_08264_gb300 import shard as SH  # noqa: E402
from paper_2503_08264_gb300 import synth as S  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


class OracleEngine:
    """The shard_forward / shard_finish pair of a shard, in FP64 on the CPU."""

    def __init__(self, sub, K, q, eps):
        self.sub, self.K, self.q, self.eps = sub, K, q, eps
        self.chain = int(getattr(sub.levels[1], "chain", 1) or 1) > 1
        self.G_own = None

    def _run(self, extra=None):
        if self.chain:
            return OC.estep(self.sub, self.q, self.K, self.eps, root_extra=extra)
        return O.estep(self.sub, self.q, self.K, self.eps, root_extra=extra)

    def shard_forward(self, q, eps, seed, it):
        r = self._run()
        n0 = self.sub.levels[0].n
        G = np.zeros((n0, self.K))
        if self.chain:
            T = self.sub.levels[1].chain
            np.add.at(G, np.asarray(self.sub.levels[1].parent)[::T], r["L"])
        else:
            np.add.at(G, np.asarray(self.sub.levels[1].parent), r["logL"][1])
        self.G_own = G
        return torch.tensor(G)

    def shard_finish(self, G):
        return self._run(G.numpy() - self.G_own)


def _models():
    return {
        "hier_logistic": (S.hier_logistic(M=23, N=5, D=3, seed=41), 16),
        "three_level": (S.batched_three_level(n_inst=2, D=2, seed=42, groups=(2, 4), units=(1, 5)), 12),
        "chain": (S.chain_poisson(n_inst=1, R=5, T=4, D=1, seed=43), 16),
    }


def _inputs(model, K):
    q = S.random_q(model, seed=7, loc_scale=0.3, sd_lo=0.3, sd_hi=0.8)
    eps = S.noise(model, K, seed=8)
    return q, eps


def _whole(model, K, q, eps):
    if int(getattr(model.levels[1], "chain", 1) or 1) > 1:
        return OC.estep(model, q, K, eps)
    return O.estep(model, q, K, eps)


def _assert_equal_fp32_tol(got_lp, got_w, got_m, ref):
    assert np.max(np.abs(got_lp - ref["log_pmp"]) / np.abs(ref["log_pmp"])) <= 1e-5
    for l in range(len(ref["w"])):
        assert got_w[l].shape == ref["w"][l].shape
        assert np.max(np.abs(got_w[l] - ref["w"][l]), initial=0.0) <= 1e-5
        scale = np.maximum(np.abs(ref["mom"][l]), 1.0)
        assert np.max(np.abs(got_m[l] - ref["mom"][l]) / scale, initial=0.0) <= 1e-5


def test_child_ranges_cover_the_plate_contiguously_and_balance_subtrees():
    model, _ = _models()["three_level"]
    for world in (1, 2, 3):
        rng = SH.child_ranges(model, world)
        assert rng[0][0] == 0 and rng[-1][1] == model.levels[1].n
        assert all(a < b for a, b in rng) and all(rng[i][1] == rng[i + 1][0] for i in range(world - 1))
    big = S.batched_three_level(n_inst=4, D=2, seed=3, groups=(5, 9), units=(1, 60))
    sizes = []
    for lo, hi in SH.child_ranges(big, 4):
        r = SH.level_ranges(big, lo, hi)
        sizes.append(sum(b - a for a, b in r[1:]))
    assert max(sizes) <= 1.5 * (sum(sizes) / 4)   # balanced by subtree, not by child count
    chain, _ = _models()["chain"]
    for lo, hi in SH.child_ranges(chain, 2):
        assert lo % 4 == 0 and hi % 4 == 0          # whole chains only
    with pytest.raises(ValueError):
        SH.child_ranges(chain, 6)                   # 5 chains for 6 ranks


def test_shard_model_remaps_parents_and_slices_data():
    model, _ = _models()["three_level"]
    lo, hi = SH.child_ranges(model, 2)[1]
    sub, ranges = SH.shard_model(model, lo, hi)
    assert ranges[0] == (0, model.levels[0].n) and ranges[1] == (lo, hi)
    g_par = np.asarray(model.levels[1].parent)
    u_par = np.asarray(model.levels[2].parent)
    a2, b2 = ranges[2]
    # every unit of the range has its group in [lo, hi), and every such unit is there
    assert set(np.nonzero((u_par >= lo) & (u_par < hi))[0]) == set(range(a2, b2))
    np.testing.assert_array_equal(np.asarray(sub.levels[1].parent), g_par[lo:hi])
    np.testing.assert_array_equal(np.asarray(sub.levels[2].parent) + lo, u_par[a2:b2])
    np.testing.assert_array_equal(sub.levels[2].y, model.levels[2].y[a2:b2])
    whole, r1 = SH.shard_model(model, 0, model.levels[1].n)
    assert [lv.n for lv in whole.levels] == [lv.n for lv in model.levels]


@pytest.mark.parametrize("name", ["hier_logistic", "three_level", "chain"])
def test_oracle_root_extra_joins_shards_into_the_whole_model(name):
    """Pin of the oracle's root_extra: two shards, each given the other's plate
    sums at the root, reproduce the whole model (Sec. 6's distributive law)."""
    model, K = _models()[name]
    q, eps = _inputs(model, K)
    ref = _whole(model, K, q, eps)
    parts, ranges_of = [], []
    engines = []
    for lo, hi in SH.child_ranges(model, 2):
        sub, ranges = SH.shard_model(model, lo, hi)
        engines.append(OracleEngine(sub, K, SH.take(q, ranges), SH.take(eps, ranges)))
        ranges_of.append(ranges)
    G = sum(e.shard_forward(None, None, 0, 0) for e in engines)
    outs = [e.shard_finish(G) for e in engines]
    for o in outs:
        np.testing.assert_allclose(o["log_pmp"], ref["log_pmp"], rtol=1e-12)
    w = SH.assemble([o["w"] for o in outs], ranges_of)
    m = SH.assemble([o["mom"] for o in outs], ranges_of)
    for l in range(len(model.levels)):
        np.testing.assert_allclose(w[l], ref["w"][l], rtol=0, atol=1e-12)
        np.testing.assert_allclose(m[l], ref["mom"][l], rtol=1e-10, atol=1e-12)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, name, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        model, K = _models()[name]
        q, eps = _inputs(model, K)
        lo, hi = SH.child_ranges(model, ws)[rank]
        sub, ranges = SH.shard_model(model, lo, hi)
        eng = OracleEngine(sub, K, SH.take(q, ranges), SH.take(eps, ranges))
        step = SH.ShardedEStep(model, K, rank, ws, engine=eng)
        assert step.ranges == ranges
        res = step.estep(None, None, 0, 0)
        gathered = [None] * ws
        dist.all_gather_object(gathered, (res["log_pmp"], res["w"], res["mom"], ranges))
        out.put((rank, gathered if rank == 0 else None))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("name", ["hier_logistic", "three_level", "chain"])
def test_gloo_world_size_2_sharded_estep_matches_single_process_oracle(name):
    ws = 2
    ctx = mp.get_context("spawn")
    q_out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, name, q_out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = dict(q_out.get(timeout=240) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = res[0]
    model, K = _models()[name]
    q, eps = _inputs(model, K)
    ref = _whole(model, K, q, eps)
    lps = [g[0] for g in gathered]
    for lp in lps[1:]:
        np.testing.assert_array_equal(lp, lps[0])     # the root step is replicated
    ranges_of = [g[3] for g in gathered]
    w = SH.assemble([g[1] for g in gathered], ranges_of)
    m = SH.assemble([g[2] for g in gathered], ranges_of)
    _assert_equal_fp32_tol(lps[0], w, m, ref)
