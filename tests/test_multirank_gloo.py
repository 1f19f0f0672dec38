"""The multi-rank host logic (q-points dealt over ranks, energies gathered) on
two gloo ranks on the CPU; the per-q work is the oracle on tiny q-points."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2405_20258_gb300.shard import qpoints_for_rank


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def sizes(iq):
    return 20 + 7 * iq, 1 + iq % 2, 4 + iq


def energy(iq):
    import oracle.rpa_oracle as orc
    from paper_2405_20258_gb300 import inputs
    n_g, n_v, n_c = sizes(iq)
    qp = inputs.make_qpoint(n_g, n_v, n_c, iq=iq, q_twentieths=inputs.qgrid_4x4x4()[iq])
    A = inputs.matrix_elements(qp)
    return orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, max(1, n_g // 4), 4)["ec"]


def worker(rank, world, port, n_q, q):
    import torch.distributed as dist
    from paper_2405_20258_gb300.shard import gather_energies
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = {iq: energy(iq) for iq in qpoints_for_rank(n_q, rank, world)}
        q.put((rank, gather_energies(local, n_q)))
    finally:
        dist.destroy_process_group()


def test_round_robin_assignment():
    assert qpoints_for_rank(5, 0, 2) == [0, 2, 4]
    assert qpoints_for_rank(5, 1, 2) == [1, 3]
    assert qpoints_for_rank(1, 0, 1) == [0]
    with pytest.raises(ValueError):
        qpoints_for_rank(4, 2, 2)


def test_two_gloo_ranks_gather_all_qpoints():
    n_q, world = 5, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, n_q, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    serial = [energy(iq) for iq in range(n_q)]
    for rank in range(world):
        assert results[rank] == pytest.approx(serial, rel=1e-12)
