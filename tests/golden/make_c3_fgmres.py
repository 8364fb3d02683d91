"""Write tests/golden/c3_oracle_fgmres.txt: the oracle's FGMRES(50) iteration
count and true residual on the 128x128x64 channelised workload (Q = own faces
+ strong A-connections, threshold 0.05), rtol 1e-8, with the digest of the
generated inputs they belong to.  Calls only the seeded generator and the
oracle (several minutes of CPU time)."""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

if __name__ == "__main__":
    t = time.time()
    s = W.config3()
    r = O.edfa_pipeline(s, mode="thresh", restart=50, rtol=1e-8, maxit=3000)
    with open(os.path.join(HERE, "c3_oracle_fgmres.txt"), "w") as f:
        f.write("# oracle FGMRES(50) on the 128x128x64 channelised workload, thresh 0.05 sets, rtol 1e-8\n")
        f.write("# written by tests/golden/make_c3_fgmres.py (oracle only)\n")
        f.write(f"inputs_sha256 {W.digest(s)}\n")
        f.write(f"iterations {r['iters']}\n")
        f.write(f"true_rel {r['true_rel']:.6e}\n")
        f.write(f"seconds {time.time() - t:.1f}\n")
