"""Multi-rank host logic on CPU with the gloo backend (world size 2): the shot
split, the fp64 gradient all-reduce of a multi-shot misfit gradient (per-shot
gradients from the fp64 oracle adjoint), timing max over ranks, whole-job rate."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2009_04619_gb300 import replicas, synth

N_SHOTS = 5


def _case():
    n_in, nb, nt = 8, 4, 24
    N = n_in + 2 * nb
    v = synth.layered_model((N, N, N), seed=7, vmin=1800, vmax=3000, perturb=0.0)
    v0 = (v * synth.gaussian_anomaly(v.shape, (N / 2, N / 2, N / 2), 2.0, -0.1)).astype(np.float32)
    vmax = float(max(v.max(), v0.max()))
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10, 10, 10)))
    go = oracle.Grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    wav = synth.ricker(nt, dt, 40.0)
    rec = synth.surface_receivers(n_in, n_in, nb, 2)
    shots = [(nb + 1 + s, nb + 2 + (s % 3), nb + 1) for s in range(N_SHOTS)]
    obs = [oracle.run_shot(go, v0, wav, nt, s, rec, want_state=False)["traces"] for s in shots]
    return go, v, wav, nt, shots, rec, obs


def _shot_fn(case):
    go, v, wav, nt, shots, rec, obs = case

    def fn(i, k=0):
        J, g = oracle.adjoint_shot(go, v, wav, nt, shots[i], rec, obs[i].astype(np.float64))
        return J, torch.from_numpy(g)
    return fn


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = _case()
        J, g = replicas.gradient_sum(_shot_fn(case), N_SHOTS, torch.zeros(case[1].shape))
        tmax = replicas.max_over_ranks(1.5 + rank)
        np.save(os.path.join(out_dir, f"g{rank}.npy"), g.numpy())
        np.save(os.path.join(out_dir, f"s{rank}.npy"), np.array([J, tmax]))
    finally:
        dist.destroy_process_group()


def test_my_shots_partition():
    for n in (0, 1, 5, 16):
        for world in (1, 2, 3, 8):
            parts = [replicas.my_shots(n, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        replicas.my_shots(4, 2, 2)


def test_job_rate():
    assert replicas.job_rate(10.0, 2.0, world=4) == 20.0
    assert replicas.job_rate([3.0, 5.0], 2.0) == 4.0


def test_gradient_sum_two_gloo_ranks_equals_one_process():
    case = _case()
    J1, g1 = replicas.gradient_sum(_shot_fn(case), N_SHOTS, torch.zeros(case[1].shape))
    assert replicas.max_over_ranks(3.25) == 3.25
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        g = [np.load(os.path.join(d, f"g{r}.npy")) for r in range(2)]
        st = [np.load(os.path.join(d, f"s{r}.npy")) for r in range(2)]
    # both ranks hold the same all-reduced result
    assert np.array_equal(g[0], g[1]) and st[0][0] == st[1][0]
    # the split sum equals the one-process sum up to fp64 reassociation
    np.testing.assert_allclose(g[0], g1.numpy(), rtol=1e-12, atol=1e-12 * np.abs(g1.numpy()).max())
    assert abs(st[0][0] - J1) <= 1e-12 * abs(J1)
    assert np.abs(g1.numpy()).max() > 0
    # timing: the slowest rank's
    assert st[0][1] == st[1][1] == 2.5


def test_gradient_sum_worker_threads_are_deterministic():
    """Two worker threads (shot i on worker i mod 2, each summing in order) give
    the same bits on every run, and the one-thread sum to fp64 reassociation."""
    case = _case()
    J1, g1 = replicas.gradient_sum(_shot_fn(case), N_SHOTS, torch.zeros(case[1].shape))
    runs = [replicas.gradient_sum(_shot_fn(case), N_SHOTS, torch.zeros(case[1].shape), workers=2)
            for _ in range(2)]
    assert runs[0][0] == runs[1][0] and torch.equal(runs[0][1], runs[1][1])
    np.testing.assert_allclose(runs[0][1].numpy(), g1.numpy(), rtol=1e-12,
                               atol=1e-12 * np.abs(g1.numpy()).max())
    assert abs(runs[0][0] - J1) <= 1e-12 * abs(J1)
