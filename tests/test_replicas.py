"""The multi-GPU replica bookkeeping (paper_0811_2518_gb300.replicas) on CPU: two gloo ranks,
each with its own unit count and time; the job rate is the units of both over the slower
rank's time.  No GPU, no CUDA extension needed (the module is plain host logic)."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
MODULE = os.path.join(HERE, "..", "paper_0811_2518_gb300", "replicas.py")


def _load():
    # the module is loaded by path: the package's __init__ needs the built CUDA library
    spec = importlib.util.spec_from_file_location("replicas_under_test", MODULE)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    R = _load().Replicas(backend="gloo")
    units = 1000.0 * (rank + 1)      # rank 0: 1000 edge-updates, rank 1: 2000
    seconds = 0.5 + 0.25 * rank      # rank 1 is the slower one
    R.barrier()
    out[rank] = (R.rank, R.world, R.max(seconds), R.sum(units), R.job_rate(units, seconds))
    R.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        rank, w, tmax, usum, rate = res[r]
        assert rank == r and w == world
        assert tmax == 0.75 and usum == 3000.0
        assert rate == pytest.approx(3000.0 / 0.75)


def test_single_process_needs_no_group():
    os.environ.pop("WORLD_SIZE", None)
    R = _load().Replicas()
    assert R.world == 1 and R.dist is None
    assert R.max(2.0) == 2.0 and R.job_rate(10.0, 2.0) == 5.0
