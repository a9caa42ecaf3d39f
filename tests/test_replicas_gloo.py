"""Replica logic of multi-GPU runs, exercised with 2 gloo ranks on the CPU.

Each rank plays one GPU: it owns a disjoint member counter range, produces per-member
results, and the host-side gather / max-over-ranks / ensemble statistics must equal the
single-process computation over all members.
"""
import math
import os
import socket

import numpy as np
import pytest

from paper_1911_03386_gb300 import replicas

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

WORLD = 2
M_PER_RANK = 6


def fake_member_results(rank):
    rng = np.random.default_rng(100 + rank)
    beta = 0.3 + 0.05 * rng.standard_normal(M_PER_RANK)
    beta[-1] = float("nan")  # a member whose run ended before the window opened
    labels = np.array([0.0, 0.4] * (M_PER_RANK // 2))
    return beta, labels


def _worker(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    beta, labels = fake_member_results(rank)
    allb = replicas.gather_members(beta, dist)
    alll = replicas.gather_members(labels, dist)
    tmax = replicas.max_over_ranks(1.5 + rank, dist)
    stats = replicas.ensemble_stats(allb, alll)
    np.save(os.path.join(out_dir, "rank%d.npy" % rank),
            np.array([tmax, stats[0.0]["mean"], stats[0.0]["se"], stats[0.4]["mean"], stats[0.4]["n"]]))
    np.save(os.path.join(out_dir, "all%d.npy" % rank), allb)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_gather_like_one_process(tmp_path):
    tmp.spawn(_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    parts = [fake_member_results(r) for r in range(WORLD)]
    allb = np.concatenate([p[0] for p in parts])
    alll = np.concatenate([p[1] for p in parts])
    ref = replicas.ensemble_stats(allb, alll)
    for r in range(WORLD):
        got = np.load(tmp_path / ("rank%d.npy" % r))
        assert got[0] == 1.5 + WORLD - 1  # max over ranks
        assert abs(got[1] - ref[0.0]["mean"]) < 1e-15 and abs(got[2] - ref[0.0]["se"]) < 1e-15
        assert abs(got[3] - ref[0.4]["mean"]) < 1e-15 and got[4] == ref[0.4]["n"] == WORLD * (M_PER_RANK // 2 - 1)
        np.testing.assert_array_equal(np.load(tmp_path / ("all%d.npy" % r)), allb)


def fake_series(rank, T=9):
    """A rank's beta series (its members x T sample times), the input of the ensemble
    moments of Sec. 3.3 Eqs. (41a,b) when the members are spread over ranks."""
    rng = np.random.default_rng(300 + rank)
    return 0.3 + 0.05 * rng.standard_normal((M_PER_RANK, T))


def _series_worker(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    allser = replicas.gather_members(fake_series(rank), dist)
    if rank == 0:
        np.save(os.path.join(out_dir, "series.npy"), allser)
    dist.barrier()
    dist.destroy_process_group()


def test_series_gathered_over_ranks_give_the_ensemble_moments(tmp_path):
    """Per-rank beta series gathered (rank order, members stacked) equal the series of the
    whole ensemble, so the moments across members over all ranks are those of one process."""
    from oracle.oracle import get as get_oracle

    tmp.spawn(_series_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    got = np.load(tmp_path / "series.npy")
    whole = np.concatenate([fake_series(r) for r in range(WORLD)], axis=0)
    np.testing.assert_array_equal(got, whole)
    orc = get_oracle()
    np.testing.assert_array_equal(orc.beta_moments(got), orc.beta_moments(whole))


def test_member_ranges_and_counter_bases():
    for m in [1, 5, 256, 1001]:
        for world in [1, 2, 3, 8]:
            ranges = [replicas.member_range(r, world, m) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == m
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    # disjoint SplitMix64 counter ranges per rank
    npts = 256 * 256
    bases = [replicas.member_counter_base(r, 256, npts) for r in range(4)]
    assert all(bases[i] + 256 * npts == bases[i + 1] for i in range(3))


def test_stats_match_textbook_formula():
    v = np.array([0.1, 0.2, 0.4, float("nan"), 0.3])
    lab = np.array([1, 1, 1, 1, 2])
    st = replicas.ensemble_stats(v, lab)
    x = np.array([0.1, 0.2, 0.4])
    assert st[1]["n"] == 3 and abs(st[1]["mean"] - x.mean()) < 1e-15
    assert abs(st[1]["se"] - math.sqrt(((x - x.mean()) ** 2).sum() / 2) / math.sqrt(3)) < 1e-15
    assert st[2]["n"] == 1 and math.isnan(st[2]["se"])
