"""Writes splitmix64_keys.txt: known answers of the random policy's draw.

The draw is the counter-based form of splitmix64 that the uniform-random
policy uses (the paper gives no policy RNG; Sec. 6 only says moves are drawn
uniformly at random):

    sm(x)      = mix(x + 0x9E3779B97F4A7C15)           one splitmix64 output
    mix(z)     : z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                 z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
    key(s, e)  = sm(sm(s) ^ e)                         per (seed, global env)
    r(s, e, p) = sm(key(s, e) ^ p)                     per ply p
    pick(r, n) = ((r >> 32) * n) >> 32                 multiply-shift index

splitmix64 is Steele, Lea and Flood, "Fast splittable pseudorandom number
generators" (OOPSLA 2014), in the form Vigna publishes.  This script is
plain Python integer arithmetic written from that definition; it imports
nothing from the oracle or the CUDA library, so the file it writes pins the
oracle's draw from outside.

    python tests/golden/make_splitmix64_keys.py   # rewrites the fixture
"""
import os

M64 = (1 << 64) - 1


def mix(z):
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & M64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def sm(x):
    return mix((x + 0x9E3779B97F4A7C15) & M64)


def key(seed, env):
    return sm(sm(seed) ^ env)


def draw(seed, env, ply):
    return sm(key(seed, env) ^ ply)


def pick(r, n):
    return ((r >> 32) * n) >> 32


# (seed, env, ply, n): the workloads' seeds, first / ragged / last env ids of
# their batches, plies from the first to beyond 64 (Reversi, Hex 11), and the
# legal counts of their first plies
CASES = [(0, 0, 0, 9), (0, 0, 1, 8), (0, 1, 0, 9), (0, 1023, 8, 1),
         (1, 0, 0, 7), (1, 65535, 41, 1), (1, 12345, 20, 5),
         (2, 0, 0, 4), (2, 262143, 59, 3), (2, 777, 64, 2),
         (3, 0, 0, 9), (3, 1048575, 120, 1), (3, 524288, 77, 44),
         (4, 65535, 3, 118), (0xFFFFFFFFFFFFFFFF, 2**40 + 3, 2**33 + 5, 121)]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "splitmix64_keys.txt")
    with open(out, "w") as f:
        f.write("# Known answers of the random policy's draw, written by make_splitmix64_keys.py\n"
                "# (plain integer arithmetic from the published splitmix64, no oracle code):\n"
                "# key = sm(sm(seed) ^ env), r = sm(key ^ ply), k = ((r >> 32) * n) >> 32.\n"
                "# Columns: seed env ply n key(hex) r(hex) k\n")
        for s, e, p, n in CASES:
            r = draw(s, e, p)
            f.write(f"{s} {e} {p} {n} {key(s, e):016x} {r:016x} {pick(r, n)}\n")
    print(out)


if __name__ == "__main__":
    main()
