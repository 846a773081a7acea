"""Word-level identities that the CUDA kernels rely on, checked in Python
integer arithmetic (no GPU, no library code involved).

Each test restates one trick of the kernels from its definition and checks it
against the plain meaning of the step it replaces:

* PT configuration moves: one pass of sequential swaps (k, k+1) for k
  ascending, applied to the 64 replica bits of a site, equals the mask-and-
  carry form ((x & starts) + sum(2^e - 2^s)) & ends plus the downward shift of
  the rest of every run.
* carry-save adder trees: the bit-planes of the count of Z one-bit words.
* the five-stage butterfly transpose of a 32 x 32 bit matrix across lanes.
* the bit-sliced butterfly that sums 32 lanes' vertical counters.
* the popcount-halving search for the rank-th set bit of a word.

The GPU parity tests check the kernels themselves; these pin the algebra that
the kernels' comments state.
"""
import random

M32 = 0xFFFFFFFF
M64 = (1 << 64) - 1


# --- PT moves -------------------------------------------------------------

def _runs(acc, n_pairs, c):
    """(start bit, end bit) of every run of accepted swaps of copy c, and the
    mask of replica bits whose configuration moves down one position."""
    runs, down = [], 0
    k = 0
    while k < n_pairs:
        if (acc >> k) & 1:
            end = k
            while end < n_pairs and (acc >> end) & 1:
                down |= 1 << (2 * end + 2 + c)
                end += 1
            runs.append((2 * k + c, 2 * end + c))
            k = end
        else:
            k += 1
    return runs, down


def _carry_moves(x, runs_by_copy, down):
    st, fw, en = [0, 0], [0, 0], [0, 0]
    for c, runs in enumerate(runs_by_copy):
        for s, e in runs:
            st[c] |= 1 << s
            en[c] |= 1 << e
            fw[c] = (fw[c] + (1 << e) - (1 << s)) & M64
    keep = ~(down | st[0] | st[1]) & M64
    y = (x & keep) | ((x & down) >> 2)
    for c in range(2):
        y |= (((x & st[c]) + fw[c]) & M64) & en[c]
    return y


def _sequential_swaps(x, accs, n_pairs):
    y = 0
    for c in range(2):
        at = list(range(n_pairs + 1))  # at[k]: the position whose configuration is now at k
        for k in range(n_pairs):
            if (accs[c] >> k) & 1:
                at[k], at[k + 1] = at[k + 1], at[k]
        for k in range(n_pairs + 1):
            y |= ((x >> (2 * at[k] + c)) & 1) << (2 * k + c)
    return y


def test_pt_moves_by_carry_equal_sequential_swaps():
    rng = random.Random(11)
    for _ in range(4000):
        n_pairs = rng.randint(1, 31)
        p = rng.random()
        accs = [sum((rng.random() < p) << k for k in range(n_pairs)) for _ in range(2)]
        r0, d0 = _runs(accs[0], n_pairs, 0)
        r1, d1 = _runs(accs[1], n_pairs, 1)
        x = rng.getrandbits(2 * (n_pairs + 1))
        assert _carry_moves(x, (r0, r1), d0 | d1) == _sequential_swaps(x, accs, n_pairs)


def test_pt_moves_all_accepted_and_none():
    for n_pairs in (1, 15, 16, 31):
        x = random.Random(n_pairs).getrandbits(2 * (n_pairs + 1))
        for accs in ((0, 0), ((1 << n_pairs) - 1, (1 << n_pairs) - 1), ((1 << n_pairs) - 1, 0)):
            r0, d0 = _runs(accs[0], n_pairs, 0)
            r1, d1 = _runs(accs[1], n_pairs, 1)
            assert _carry_moves(x, (r0, r1), d0 | d1) == _sequential_swaps(x, accs, n_pairs)


# --- carry-save counts ----------------------------------------------------

def _full_add(a, b, c):
    x = a ^ b
    return x ^ c, (a & b) | (c & x)


def _csa_count(x):
    z = len(x)
    a, ca = _full_add(x[0], x[1], x[2])
    if z == 4:
        h = a & x[3]
        return a ^ x[3], ca ^ h, ca & h, 0
    b, cb = _full_add(x[3], x[4], x[5])
    if z == 6:
        c1, c2 = _full_add(ca, cb, a & b)
        return a ^ b, c1, c2, 0
    c, cc = _full_add(a, b, x[6])
    h = c & x[7]
    t, e = _full_add(ca, cb, cc)
    f = t & h
    return c ^ x[7], t ^ h, e ^ f, e & f


def test_carry_save_counts_every_bit_pattern():
    for z in (4, 6, 8):
        # bit b of the inputs enumerates all 2^z patterns over the bit lanes
        for base in range(0, 1 << z, 32):
            x = [0] * z
            for b in range(32):
                pat = (base + b) % (1 << z)
                for d in range(z):
                    x[d] |= ((pat >> d) & 1) << b
            planes = _csa_count(x)
            for b in range(32):
                pat = (base + b) % (1 << z)
                got = sum(((planes[i] >> b) & 1) << i for i in range(4))
                assert got == bin(pat).count("1")


# --- warp transposes and sums -----------------------------------------------

_TRANSPOSE_MASK = {16: 0x0000FFFF, 8: 0x00FF00FF, 4: 0x0F0F0F0F, 2: 0x33333333, 1: 0x55555555}


def _warp_transpose(rows):
    x = list(rows)
    for s in (16, 8, 4, 2, 1):
        m = _TRANSPOSE_MASK[s]
        o = [x[lane ^ s] for lane in range(32)]  # every lane reads before any writes
        x = [((x[l] & ~m & M32) | ((o[l] >> s) & m)) if l & s else ((x[l] & m) | ((o[l] << s) & ~m & M32))
             for l in range(32)]
    return x


def test_warp_bit_transpose():
    rng = random.Random(5)
    for _ in range(200):
        a = [rng.getrandbits(32) for _ in range(32)]
        t = _warp_transpose(a)
        for j in range(32):
            assert t[j] == sum(((a[l] >> j) & 1) << l for l in range(32))


def _warp_vsum(planes_by_lane, npl):
    a = [list(p) + [0] * 5 for p in planes_by_lane]
    for st in range(5):
        s = 16 >> st
        old = [row[:] for row in a]
        for lane in range(32):
            cy = 0
            for i in range(npl + st):
                o = old[lane ^ s][i]
                x = old[lane][i] ^ o
                ncy = (old[lane][i] & o) | (cy & x)
                a[lane][i] = x ^ cy
                cy = ncy
            a[lane][npl + st] = cy
    return [sum(((a[lane][i] >> lane) & 1) << i for i in range(npl + 5)) for lane in range(32)]


def test_bit_sliced_warp_sum_up_to_full_counters():
    rng = random.Random(9)
    for npl in (4, 8):
        for trial in range(30):
            top = (1 << npl) - 1
            counts = [[top if trial == 0 else rng.randint(0, top) for _ in range(32)] for _ in range(32)]
            planes = [[sum(((counts[l][b] >> i) & 1) << b for b in range(32)) for i in range(npl)] for l in range(32)]
            got = _warp_vsum(planes, npl)
            assert got == [sum(counts[l][b] for l in range(32)) for b in range(32)]


# --- rank-th set bit --------------------------------------------------------

def _nth_set_bit(w, rank):
    pos = 0
    for hw in (16, 8, 4, 2, 1):
        lo = w & ((1 << hw) - 1)
        cl = bin(lo).count("1")
        if rank >= cl:
            rank -= cl
            w >>= hw
            pos += hw
        else:
            w = lo
    return pos


def test_rank_th_set_bit():
    rng = random.Random(3)
    words = [M32, 1, 1 << 31, 0x80000001] + [rng.getrandbits(32) & rng.getrandbits(32) for _ in range(3000)]
    for w in words:
        bits = [i for i in range(32) if (w >> i) & 1]
        for r, b in enumerate(bits):
            assert _nth_set_bit(w, r) == b


def test_pt_moves_need_one_carry_per_copy():
    """The runs of the two copies interleave bit by bit, so one addition over
    both copies' runs at once lets a carry of one copy cross the other's
    run: the per-copy split is needed."""
    rng = random.Random(17)
    differs = 0
    for _ in range(2000):
        n_pairs = rng.randint(2, 31)
        accs = [rng.getrandbits(n_pairs) for _ in range(2)]
        r0, d0 = _runs(accs[0], n_pairs, 0)
        r1, d1 = _runs(accs[1], n_pairs, 1)
        x = rng.getrandbits(2 * (n_pairs + 1))
        merged = _carry_moves(x, (r0 + r1, []), d0 | d1)
        differs += merged != _sequential_swaps(x, accs, n_pairs)
    assert differs > 0
