"""E over every node of the N = M = 2^20 Fourier-Laplace workload (not a test
module: a checker run by hand on the host cores, about an hour on 8 cores).

E = max_j |f_j - f~_j| / sum_k |c_k| (the error measure of Section 5) of a saved
GPU result against the oracle's FP64 direct sum at all M nodes, where the
bench's and the tests' samples cover a few thousand.  The result comes from

    python bench.py --case flt_2e20_fp32 --steps 1 --warmup 1 --save f_fp32.npy
    python bench.py --case flt_2e20_fp64ff --steps 1 --warmup 1 --save f_ff.npy

and is checked with

    python tests/full_error.py f_fp32.npy f_ff.npy --cache ref_2e20.npy

The oracle's values are computed in chunks of 2^15 nodes and kept in the cache
file, so an interrupted run resumes where it stopped.
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402  (the seeded workload of the bench)
import oracle  # noqa: E402


def reference(c, w, cache, chunk=1 << 15):
    M = w.shape[0]
    ref = np.load(cache) if cache and os.path.exists(cache) else np.full(M, np.nan, dtype=np.complex128)
    if ref.shape != (M,):
        raise ValueError(f"{cache}: {ref.shape[0]} values for {M} nodes")
    t0 = time.time()
    for s in range(0, M, chunk):
        if not np.isnan(ref[s].real):
            continue
        ref[s:s + chunk] = oracle.flt_direct(c, w[s:s + chunk], threads=oracle.default_threads())
        if cache:
            np.save(cache, ref)
        print(f"oracle: {min(s + chunk, M)}/{M} nodes, {time.time() - t0:.0f} s", flush=True)
    return ref


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("outputs", nargs="+", help=".npy results saved by bench.py --case ... --save")
    ap.add_argument("--N", type=int, default=1 << 20, help="workload size N = M (default 2^20)")
    ap.add_argument("--cache", default=None, help=".npy file holding the oracle's values (resumable)")
    args = ap.parse_args()
    c64, w = bench.rank_workload(args.N, 0)
    c = c64.astype(np.complex128)
    ref = reference(c, w, args.cache)
    cs = np.sum(np.abs(c))
    for path in args.outputs:
        f = np.load(path).astype(np.complex128)
        err = np.abs(f - ref)
        j = int(np.argmax(err))
        print(f"{os.path.basename(path)}: E over all {len(f)} nodes = {err[j] / cs:.3e} "
              f"(worst node {j}, |f| there {abs(ref[j]):.3g}); oracle on {oracle.default_threads()} cores",
              flush=True)


if __name__ == "__main__":
    main()
