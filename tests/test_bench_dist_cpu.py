"""Multi-rank host logic of bench.py on the CPU: two gloo ranks (rendezvous on
127.0.0.1) run the set-up, barrier and max-over-ranks reduction that the
timed region uses, and the reference arm's non-zero rank returns without
work (rank 0 alone times and prints it)."""
import os
import socket
import subprocess
import sys
import textwrap

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_barrier_max_and_reference_ranks(tmp_path):
    script = tmp_path / "rank.py"
    script.write_text(textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import bench

        class Args:
            pass

        rank, world, local, pg = bench.dist_setup(Args())
        bench.barrier(pg)
        m = bench.max_over_ranks(pg, 1.5 + rank)
        ref = bench.run_reference(Args(), rank, world) if rank != 0 else "skipped"
        bench.barrier(pg)
        print("RESULT", rank, world, m, ref, flush=True)
        pg.destroy_process_group()
    """ % REPO))
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=240)[0] for p in procs]
    for rank, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        line = [l for l in out.splitlines() if l.startswith("RESULT")][-1].split()
        assert line[1:5] == [str(rank), "2", "2.5", "skipped" if rank == 0 else "None"], line
