"""The row partition of the distributed setting (Section 3, Section 5.3) on CPU
ranks: the library's host-side partition and halo plan (bcs_partition_rows,
bcs_halo_plan) drive a row-partitioned run of the oracle on two gloo ranks,
each owning one block of rows of every vector.  Before every matrix-vector
product a rank sends the values its send list names and receives its halo;
every inner product is the exact sum of the ranks' exact partials, rounded
once.  The run must reproduce the single-process oracle bit for bit."""
import os
import socket

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bcs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2108_10591_gb300 as m
    return m


def _matrices():
    return [W.cd2d(20, 20.0), W.powerlaw(n=3001, seed=5), W.cd3d_upwind(10, 50.0)]


def test_partition_rows_is_balanced(bcs):
    for A in _matrices():
        w = np.diff(A.rowptr) + 1                       # weight of a row: its nonzeros + 1
        for p in [1, 2, 3, 7, 16]:
            bd = bcs.partition_rows(A, p)
            assert bd[0] == 0 and bd[-1] == A.n and np.all(np.diff(bd) >= 0)
            blocks = np.array([w[bd[k]:bd[k + 1]].sum() for k in range(p)])
            assert blocks.max() - w.sum() / p <= w.max()   # within one row of the even share
    A = W.cd2d(2, 1.0)                                    # fewer rows than ranks: empty blocks allowed
    bd = bcs.partition_rows(A, 7)
    assert bd[-1] == 4 and np.all(np.diff(bd) >= 0)
    with pytest.raises(bcs.BcsError):
        bcs.partition_rows(A, 17)


def _extended(plan, x_global):
    """The rank's extended vector (left halo, its rows padded to npad, right halo) built from
    every rank's send list applied to x_global -- what the halo exchange delivers."""
    nl, npad = len(plan["left"]), plan["npad"]
    ext = np.full(nl + npad + len(plan["right"]), np.nan)
    ext[nl:nl + plan["nloc"]] = x_global[plan["row0"]:plan["row0"] + plan["nloc"]]
    return ext


def test_halo_plans_deliver_every_halo_entry_once(bcs, orc):
    rng = np.random.default_rng(3)
    for A in _matrices():
        xg = rng.standard_normal(A.n)
        yg = orc.spmv(A, xg)
        for p in [1, 2, 3, 5]:
            bd = bcs.partition_rows(A, p)
            plans = [bcs.halo_plan(A, bd, r) for r in range(p)]
            exts = [_extended(pl, xg) for pl in plans]
            hits = [np.zeros(len(e), dtype=int) for e in exts]
            for src, pl in enumerate(plans):
                for row, q, off in zip(pl["send_row"], pl["send_rank"], pl["send_off"]):
                    assert q != src
                    k = len(plans[q]["left"]) + off
                    exts[q][k] = xg[pl["row0"] + row]
                    hits[q][k] += 1
            for r, pl in enumerate(plans):
                nl = len(pl["left"])
                halo = np.r_[np.arange(nl), nl + pl["npad"] + np.arange(len(pl["right"]))]
                assert np.all(hits[r][halo] == 1)                      # every halo entry exactly once
                assert np.array_equal(exts[r][halo], xg[np.r_[pl["left"], pl["right"]]])
                # the block's rows of A x from its local columns, bit for bit (same CSR order)
                r0, r1 = bd[r], bd[r + 1]
                rp = A.rowptr[r0:r1 + 1] - A.rowptr[r0]
                loc = W.CSR(pl["nloc"], rp, (pl["local_col"] + nl).astype(np.int32),
                            A.val[A.rowptr[r0]:A.rowptr[r1]])
                yl = orc.spmv(loc, exts[r]) if pl["nloc"] else np.zeros(0)
                assert np.array_equal(yl, yg[r0:r1])


# ---- two gloo ranks ------------------------------------------------------------------------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, cases, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    import paper_2108_10591_gb300 as bcs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    try:
        for name, kind, kw in cases:
            A = {"cd2d": lambda: W.cd2d(24, 20.0), "powerlaw": lambda: W.powerlaw(n=2999, seed=11)}[name]()
            b = W.rhs_ones(A)
            bd = bcs.partition_rows(A, world)
            pl = bcs.halo_plan(A, bd, rank)
            r0, r1, nl, npad = pl["row0"], pl["row0"] + pl["nloc"], len(pl["left"]), pl["npad"]
            loc = W.CSR(pl["nloc"], A.rowptr[r0:r1 + 1] - A.rowptr[r0], (pl["local_col"] + nl).astype(np.int32),
                        A.val[A.rowptr[r0]:A.rowptr[r1]])
            ext = np.zeros(nl + npad + len(pl["right"]))
            stats = {"mv": 0, "dot": 0, "sent": 0}

            def mv(x, y):
                # halo exchange: every rank's (offset, value) pairs for every other rank
                msg = {}
                for qq in range(world):
                    sel = pl["send_rank"] == qq
                    msg[qq] = (pl["send_off"][sel], x[pl["send_row"][sel]].copy())
                got = [None] * world
                dist.all_gather_object(got, msg)
                ext[nl:nl + pl["nloc"]] = x
                for src in range(world):
                    if src != rank:
                        off, val = got[src][rank]
                        ext[nl + off] = val
                y[:] = oracle.spmv(loc, ext)
                stats["mv"] += 1
                stats["sent"] += int(sum(len(v[1]) for k_, v in msg.items() if k_ != rank))

            def dot(x, y):
                limbs, ok = oracle.dot_partial(x, y)
                got = [None] * world
                dist.all_gather_object(got, (limbs, ok, float(np.dot(x, y))))
                stats["dot"] += 1
                if all(g[1] for g in got):
                    return oracle.dot_round(oracle.dot_merge([g[0] for g in got]))
                return sum(g[2] for g in got)   # a non-finite operand: propagate it

            res = oracle.solve_hooked(pl["nloc"], b[r0:r1], mv, dot, kind=kind, **kw)
            xs = [None] * world
            dist.all_gather_object(xs, res["x"])
            out.append((name, kind, res["iterations"], res["restarts"], res["rr_steps"], res["hist"],
                        np.concatenate(xs), stats))
        q.put((rank, out, None))
    except Exception as e:  # noqa: BLE001
        q.put((rank, None, repr(e)))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_row_partitioned_oracle(bcs, orc):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    cases = [("cd2d", "p-BiCGSafe", dict(tol=1e-10, maxit=600, max_restarts=9)),
             ("cd2d", "ssBiCGSafe2", dict(tol=1e-10, maxit=600, max_restarts=9)),
             ("cd2d", "p-BiCGSafe-rr", dict(tol=1e-10, maxit=600, rr_m=9, max_restarts=9)),
             ("powerlaw", "p-BiCGSafe-rr", dict(tol=1e-10, maxit=600, rr_m=20, max_restarts=9))]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, cases, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(2):
        rank, out, err = q.get(timeout=300)
        assert err is None, err
        got[rank] = out
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for k, (name, kind, kw) in enumerate(cases):
        A = {"cd2d": lambda: W.cd2d(24, 20.0), "powerlaw": lambda: W.powerlaw(n=2999, seed=11)}[name]()
        b = W.rhs_ones(A)
        ref = orc.solve(A, b, kind=kind, **kw)
        assert ref["status"] == 0
        for rank in range(2):
            _, _, its, rst, rr, hist, x, stats = got[rank][k]
            assert its == ref["iterations"] and rst == ref["restarts"] and rr == ref["rr_steps"]
            assert np.array_equal(hist, ref["hist"])
            assert np.array_equal(x, ref["x"])
            assert stats["sent"] > 0 and stats["dot"] > 0
