"""Write tests/golden/c3_oracle_fgmres.txt: the oracle's FGMRES(50) iteration
counts and true residuals on the 128x128x64 channelised workload (Q = own
faces + strong A-connections, threshold 0.05), rtol 1e-8, with the natural
order of the inner ILU(0) factorisations, with multicolour orderings of both
(ordering 2) and with the block multicolour ordering of S~ (blocks of 4 rows),
the residual estimates of the first restart cycle of
each, and the digest of the generated inputs they belong to.
Calls only the seeded generator and the oracle (tens of minutes of CPU
time)."""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

if __name__ == "__main__":
    s = W.config3()
    out = []
    for ordering, blk, suffix in ((0, 1, ""), (2, 1, "_ordering2"), (2, 4, "_ordering2_block4")):
        t = time.time()
        r = O.edfa_pipeline(s, mode="thresh", restart=50, rtol=1e-8, maxit=3000, ordering=ordering, s_block=blk)
        out.append((suffix, r["iters"], r["true_rel"], time.time() - t, r["hist"][1:51]))
    with open(os.path.join(HERE, "c3_oracle_fgmres.txt"), "w") as f:
        f.write("# oracle FGMRES(50) on the 128x128x64 channelised workload, thresh 0.05 sets, rtol 1e-8\n")
        f.write("# (natural order; _ordering2: multicolour orderings of A~ and S~; _block4: S~ in blocks of 4 rows)\n")
        f.write("# written by tests/golden/make_c3_fgmres.py (oracle only)\n")
        f.write(f"inputs_sha256 {W.digest(s)}\n")
        for suffix, it, tr, sec, hist in out:
            f.write(f"iterations{suffix} {it}\n")
            f.write(f"cycle1{suffix} " + " ".join(f"{v:.17e}" for v in hist) + "\n")
            f.write(f"true_rel{suffix} {tr:.6e}\n")
            f.write(f"seconds{suffix} {sec:.1f}\n")
