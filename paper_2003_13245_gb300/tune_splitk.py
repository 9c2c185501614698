"""Tile tuner of the tensor-core contractions (run on the GPU; writes the table the library
reads).

Every contraction of the mixed-precision path is one tcgen05 GEMM of shape (M, N, K) summed over
nred operand pairs for nbatch outputs, computed in 128-row tiles of 64 or 128 columns; when the
output has few tiles its K loop is split over CTAs and a second kernel adds the partial sums.
This script runs short versions of the benchmark workloads with shape recording on (the
contraction shapes depend only on the local dimensions, the bond dimensions and the MPO bond
dimension, so four molecules per chain give every bulk shape of a long chain), times every
recorded shape at each candidate (tile width, split), and writes the fastest per shape to
tc_splitk_table.txt beside libtdmrg.so:

    python -m paper_2003_13245_gb300.tune_splitk [--out PATH] [--reps 10]
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CANDIDATES = [1, 2, 3, 4, 6, 8, 12, 16, 24, 32]

# (label, N, omega, g, nmax, V, peierls, M): the chains of the benchmark workloads, shortened
WORKLOADS = [
    ("two-mode chain, M=128", 4, [0.2, 1.0], [1.5, 0.8], [8, 4], 0.5, None, 128),
    ("two-mode chain, M=96", 4, [0.2, 1.0], [1.5, 0.8], [6, 4], 1.0, None, 96),
    ("two-mode chain, M=64", 4, [0.2, 1.0], [1.5, 0.8], [6, 4], 0.5, None, 64),
] + [("one-mode chain, M=%d" % M, 4, [1.0], [1.0], [6], 1.0, None, M)
     for M in (32, 48, 64, 96, 128)] + [
    ("Holstein-Peierls chain, M=64", 4, [0.2, 1.0], [1.5, 0.8], [4, 3], 1.0, (0.1, 0.2, 8), 64),
]


def record_shapes():
    from paper_2003_13245_gb300 import Model, PREC_C64_3XTF32, binding
    shapes = set()
    for label, N, om, g, nm, V, peierls, M in WORKLOADS:
        binding.tune_record_shapes(True)
        m = Model(N, om, g, nm, V, peierls=peierls, precision=PREC_C64_3XTF32)
        try:
            m.thermal_prepare(0.1, 0.05, M)
            m.realtime_init()
            m.realtime_step(1, 0.05)
            m.realtime_observe()
        finally:
            m.close()
        got = binding.tune_recorded_shapes()
        binding.tune_record_shapes(False)
        print("%-32s %d shapes" % (label, len(got)), flush=True)
        shapes.update(got)
    return sorted(shapes)


def tune(shapes, reps):
    from paper_2003_13245_gb300 import binding
    rows = []
    for (M, N, K, nred, nbatch) in shapes:
        kt = ((K + 15) // 16) * nred
        best = None
        for bn in ((64, 128) if N > 64 else (64,)):
            for ks in CANDIDATES:
                if ks > kt:
                    break
                ms = binding.kernel_tc_gemm_timed(M, N, K, nred, nbatch, ks, reps, tile_n=bn)
                if best is None or ms < best[1]:
                    best = (ks, ms, bn)
        rule = binding.kernel_tc_gemm_timed(M, N, K, nred, nbatch, 0, reps, tile_n=64)
        rows.append((M, N, K, nred, nbatch, best[0], best[1], rule, best[2]))
        print("%6d %6d %5d %3d %3d  split %2d  tile %3d  %.4f ms  (rule %.4f ms)" %
              (M, N, K, nred, nbatch, best[0], best[2], best[1], rule), flush=True)
    return rows


def main():
    import torch
    from paper_2003_13245_gb300 import binding
    from paper_2003_13245_gb300.build import LIB, build_library
    p = argparse.ArgumentParser()
    p.add_argument("--out", default=os.path.join(os.path.dirname(LIB), "tc_splitk_table.txt"))
    p.add_argument("--reps", type=int, default=10)
    a = p.parse_args()
    build_library()
    if not torch.cuda.is_available():
        raise SystemExit("tune_splitk needs a CUDA GPU")
    os.environ["TDMRG_SPLITK_TABLE"] = os.devnull     # record and time without a table
    binding.tune_reload_table()
    rows = tune(record_shapes(), a.reps)
    name = torch.cuda.get_device_name(0)
    with open(a.out, "w") as f:
        f.write("# tile table of the tensor-core contractions, measured on %s by "
                "tune_splitk.py\n# M N K nred nbatch ksplit tile_n   (best ms, ms of 64-column "
                "tiles with the occupancy rule)\n" % name)
        for M, N, K, r, b, ks, ms, rule, bn in rows:
            f.write("%d %d %d %d %d %d %d   # %.4f %.4f\n" % (M, N, K, r, b, ks, bn, ms, rule))
    gain = sum(r[7] for r in rows) / max(sum(r[6] for r in rows), 1e-30)
    print("wrote %s (%d shapes; summed time of the rule / of the table: %.3f)" %
          (a.out, len(rows), gain))


if __name__ == "__main__":
    main()
