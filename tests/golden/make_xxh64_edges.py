"""Write xxh64_edges.txt: XXH64 of a fixed byte pattern at every length that
takes a different path through the algorithm, from the oracle alone.

The digest of the hot path is XXH64 with seed 0 of each page's bytes (the
paper hashes captured regions page by page); XXH64 is defined by the public
xxHash specification.  The lengths cover every tail path (0..70: no stripe,
partial stripe, 8-byte, 4-byte and single-byte tails), stripe edges and page
edges, at seed 0 and at three other seeds.  The values are computed by the
oracle only; test_oracle_digest.py checks them against the system's
libxxhash where it is installed, and the GPU tests check kc_digest against
them where it is not.

Run from the repository root:  python tests/golden/make_xxh64_edges.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

LENGTHS = (list(range(0, 71)) + [95, 96, 97, 127, 128, 129, 255, 256, 257, 1000,
                                 4095, 4096, 4097, 65535, 65536, 65537])
SEEDS = (0, 1, 0x9E3779B97F4A7C15, 2**64 - 1)


def pattern(n: int) -> bytes:
    """Byte i = (i * 131 + 7) mod 251: no zero runs, no period of 2^k."""
    return bytes((i * 131 + 7) % 251 for i in range(n))


def main() -> None:
    out = os.path.join(HERE, "xxh64_edges.txt")
    with open(out, "w") as f:
        f.write("# XXH64 (public xxHash specification) of pattern(len), byte i = (i*131+7) mod 251.\n")
        f.write("# Written by tests/golden/make_xxh64_edges.py from the oracle; columns: len seed hash (hex).\n")
        for seed in SEEDS:
            for n in LENGTHS:
                f.write(f"{n} {seed:#x} {oracle.xxh64(pattern(n), seed):#018x}\n")


if __name__ == "__main__":
    main()
