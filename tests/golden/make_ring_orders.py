"""Write the oracle's greedy ring orderings (Sec. III-E) for the large band-limits of the tests.

Calls only oracle/.  Output: tests/golden/ring_order_L{L}.txt, one index t per line, k = 0..L-1,
theta_k = pi (2 t + 1) / (2 L - 1) (Eq. (19)).  The orderings are stored because the oracle's
O(L^4) planner takes minutes at these L; the paper likewise computes them once per L and stores
them (Sec. III-E).

    python tests/golden/make_ring_orders.py 512 1024
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from oracle.sampling import greedy_order_secular  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

if __name__ == "__main__":
    for arg in sys.argv[1:]:
        L = int(arg)
        t0 = time.time()
        order = greedy_order_secular(L)
        path = os.path.join(HERE, f"ring_order_L{L}.txt")
        with open(path, "w") as f:
            f.write(f"# greedy ring ordering, L={L}, oracle.sampling.greedy_order_secular\n")
            f.write("\n".join(str(int(t)) for t in order) + "\n")
        print(f"L={L}: {time.time() - t0:.1f} s -> {path}", flush=True)
