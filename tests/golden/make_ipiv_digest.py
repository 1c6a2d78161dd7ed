"""Write the pivot-vector digest of the FP64 LU at the benchmark size.

Factors the n x n matrix of generator stream 0 under the given seed with the
CPU oracle's LU with partial pivoting (LAPACK dgetf2 semantics: first largest
|a_ik| wins, full-row interchanges; Sec. III-A.1 of the paper), then records
the SHA-256 of the 0-based int32 pivot vector (little-endian bytes), the
number of interchanges, the smallest relative gap between the two largest
pivot candidates of any column, and the first pivots in plain text. Only the
oracle is called; the GPU test compares its own pivot vector with this file.

    python tests/golden/make_ipiv_digest.py [n] [seed]     # default 32768 1

At n = 32768 this takes about an hour on 8 x86 cores (the oracle is the
unblocked elimination, bound by memory bandwidth).
"""
import hashlib
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 32768
    seed = int(sys.argv[2]) if len(sys.argv) > 2 else 1
    t0 = time.time()
    A = oracle.generate(seed, oracle.STREAM_A, n, n)
    _, ipiv, info, gap = oracle.getrf(A)
    dt = time.time() - t0
    del A
    digest = hashlib.sha256(np.ascontiguousarray(ipiv, dtype="<i4").tobytes()).hexdigest()
    swaps = int(np.count_nonzero(ipiv != np.arange(n, dtype=np.int32)))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"ipiv_n{n}_seed{seed}.txt")
    with open(out, "w") as f:
        f.write(f"# Pivot vector of the oracle's LU with partial pivoting, n = {n}, seed = {seed},\n")
        f.write("# matrix of generator stream 0 (uniform[-0.5, 0.5) entries). Written by\n")
        f.write("# tests/golden/make_ipiv_digest.py from the oracle alone "
                f"({oracle.num_threads()} threads, {dt:.0f} s).\n")
        f.write(f"n {n}\nseed {seed}\ninfo {info}\n")
        f.write(f"sha256_ipiv_int32_le {digest}\n")
        f.write(f"interchanges {swaps}\n")
        f.write(f"min_gap {gap!r}\n")
        f.write("first64 " + " ".join(str(int(v)) for v in ipiv[:64]) + "\n")
        f.write("last64 " + " ".join(str(int(v)) for v in ipiv[-64:]) + "\n")
    print(out, digest, gap, dt)


if __name__ == "__main__":
    main()
