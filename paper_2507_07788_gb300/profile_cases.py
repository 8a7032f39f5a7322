"""Small, self-contained workloads that exercise each kernel of the library,
for per-kernel profiling (ncu -k <kernel> -s <skip> -c <count> python -m
paper_2507_07788_gb300.profile_cases <case> ...).  Inputs are the seeded
synthetic matrices of paper_2507_07788_gb300.synth; every case runs its
calls `--reps` times and synchronizes at the end.

Cases:
  factor   cholqr_factor of an m x n matrix with condition number kappa
           (--emulation auto|off|tcgen05, --precision fp64|mixed)
  gram     cholqr_gram of the same matrix (--precision fp64|mixed)
  append   a basis of q columns (appends of --p), then --reps appends of p
           columns; --cache enables the digit cache of the basis
  serve    small appends to several bases through the serving runtime
           (batched kernels)
  sharded  cholqr_factor_sharded with two simulated ranks on one device
"""
from __future__ import annotations

import argparse
import sys
import threading


def _parse(argv):
    ap = argparse.ArgumentParser(prog="python -m paper_2507_07788_gb300.profile_cases")
    ap.add_argument("case", choices=["factor", "gram", "append", "serve", "sharded"])
    ap.add_argument("--m", type=int, default=300000)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--kappa", type=float, default=1e12)
    ap.add_argument("--q", type=int, default=64)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--cache", action="store_true")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--emulation", choices=["auto", "off", "tcgen05"], default="auto")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    return ap.parse_args(argv)


def main(argv=None) -> int:
    args = _parse(sys.argv[1:] if argv is None else argv)
    import torch

    import paper_2507_07788_gb300 as cq
    from paper_2507_07788_gb300 import synth

    emu = {"auto": cq.EMU_AUTO, "off": cq.EMU_OFF, "tcgen05": cq.EMU_TCGEN05}[args.emulation]
    prec = {"fp64": cq.PREC_FP64, "mixed": cq.PREC_MIXED}[args.precision]
    opts = cq.default_opts(emulation=emu, precision=prec)
    m, n = args.m, args.n
    if args.case in ("factor", "gram", "sharded"):
        A = cq.to_colmajor(synth.test_matrix(m, n, args.kappa, rep=0))
        if args.case == "factor":
            Q, R = cq.colmajor(m, n), cq.colmajor(n, n)
            for _ in range(args.reps):
                res = cq.factor(A, Q=Q, R=R, opts=opts, check=False)
                assert res.status == cq.OK, res.info
        elif args.case == "gram":
            for _ in range(args.reps):
                cq.gram(A, opts=opts)
        else:
            from paper_2507_07788_gb300.sharded import LocalReducerGroup, factor_sharded, split_rows
            world = 2
            grp = LocalReducerGroup(world, n * n, timeout_s=60.0)
            blocks = split_rows(m, world)
            shards = [cq.to_colmajor(A[r0:r1]) for r0, r1 in blocks]
            torch.cuda.synchronize()
            for _ in range(args.reps):
                out = [None] * world

                def rank_main(r):
                    s = torch.cuda.Stream()
                    with torch.cuda.stream(s):
                        out[r] = factor_sharded(shards[r], m, grp.reducer(r), opts=opts, stream=s, check=False)
                    s.synchronize()

                th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
                for t in th:
                    t.start()
                for t in th:
                    t.join()
                assert all(o.status == cq.OK for o in out), [o.status for o in out]
    elif args.case == "append":
        q, p = args.q, args.p
        b = cq.Basis(m, q + p * args.reps, opts=opts)
        if args.cache:
            b.enable_digit_cache()
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        blk = torch.randn((q, m), generator=gen, device="cuda", dtype=torch.float64).t()
        st, _ = b.append(blk)
        assert st == cq.OK, st
        for _ in range(args.reps):
            N = torch.randn((p, m), generator=gen, device="cuda", dtype=torch.float64).t()
            st, _ = b.append(N)
            assert st == cq.OK, st
        b.close()
    else:  # serve: small appends, batched
        srv = cq.Server(slots=4, batch_max=16, hbm_budget_bytes=1 << 30, small_rows=262144)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(11)
        bases = [cq.Basis(min(m, 200000), 64) for _ in range(8)]
        tickets = []
        for _ in range(args.reps):
            for b in bases:
                N = torch.randn((args.p, b.m), generator=gen, device="cuda", dtype=torch.float64).t()
                tickets.append(srv.submit_append(b, N))
        for t in tickets:
            assert srv.wait(t)["status"] >= 0
        srv.close()
        for b in bases:
            b.close()
    torch.cuda.synchronize()
    print("profile case done:", args.case, f"m={m} n={n}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
