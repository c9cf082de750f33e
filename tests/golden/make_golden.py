"""Writes the stored expected values under tests/golden/ by running ONLY the oracle (dense FP64
HKM PDIPM, oracle/pdipm.py) on the seeded workloads from instances/.  Nothing here touches the
CUDA path.  Usage: python tests/golden/make_golden.py [workload ...]"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from instances import workload  # noqa: E402
from instances import sdpa  # noqa: E402
from oracle.sdp import SparseSym  # noqa: E402
from oracle import pdipm  # noqa: E402


def main(names):
    for name in names:
        inst = workload(name)
        A = SparseSym.from_instance(inst)
        t = time.time()
        res = pdipm.solve_dense(A, inst.b, inst.z0,
                                log=lambda h: print(name, h, flush=True))
        out = dict(workload=name, n=inst.n, m=inst.m,
                   instance_sha256=sdpa.content_hash(sdpa.to_text(inst)),
                   status=res["status"], pobj=res["pobj"],
                   dobj=res["dobj"], gap=res["gap"], pinf=res["pinf"], dinf=res["dinf"],
                   iters=res["iters"], seconds=time.time() - t,
                   source="oracle.pdipm.solve_dense (dense FP64 HKM PDIPM, beta 0.1, gamma 0.9, "
                          "tol 1e-7), tests/golden/make_golden.py")
        with open(os.path.join(ROOT, "tests", "golden", f"{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(out, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["block_arrow_1020", "block_arrow_2020"])
