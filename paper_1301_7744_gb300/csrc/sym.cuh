// sym.cuh — symmetry inside diagonal blocks (host + device).
//
// BCSS stores every unique block in full, the diagonal ones (repeated block
// indices) included, and the paper's algorithm computes every entry of such
// a block (Sec. 3.3 and 5.3 leave the symmetry inside a block unused).  The
// temporary T^(k) is symmetric in its k leading modes (the i modes not yet
// contracted) and in its m - k trailing modes (the j modes already
// produced), Sec. 5.3.  Inside a stored block of T^(k) an entry is therefore
// equal to the one whose full indices are non-decreasing within each of the
// two groups: its canonical entry.  A level run in the in-block-symmetry mode
// computes the canonical entries only; a temporary keeps just those (the next
// level reads every operand entry at its canonical position), and the level
// that writes the call's result copies each to every position of its block
// that equals it by symmetry, so C keeps the BCSS layout with full blocks.
// Per level the canonical entries are the unique entries of T^(k),
// C(n + k - 1, k) C(p + m - k - 1, m - k) when b divides n and p, which makes
// the flop count the minimum of Sec. 6 ("analysis relative to minimum").
//
// Canonical rows of a parent node (level d, k = m - 1 - d; modes 0 .. k-1 hold
// the sorted i blocks I_0 <= ... <= I_{k-1}, mode k the new j block (the
// tile's column), modes k+1 .. m-1 the parent's j blocks u_0 <= ... <=
// u_{d-1}) are enumerated by rho = rho_i + N_i rho_j:
//   rho_i = colex rank of the non-decreasing tuple of full i indices
//           x_0 <= ... <= x_{k-1} over [0, nbar b)  (N_i = C(nbar b + k - 1, k)),
//           giving the block tuple I_t = x_t / b and offsets x_t mod b;
//   rho_j = mixed radix over the runs of equal parent blocks, each run of
//           length g a colex-ranked non-decreasing g-tuple of offsets in
//           [0, b) (C(b + g - 1, g) values).
// A column c of child block jb is canonical unless jb = u_0 (the diagonal
// child, which joins the run of u_0) and c exceeds the offset of mode k+1.
#pragma once

#include "common.cuh"

constexpr int SYM_V = 65;   // table columns: values 0 .. 64 (nbar b <= 64 and b <= 64)
constexpr int SYM_T = 4;    // table rows: positions 0 .. 3 (orders m <= 5: at most 4 modes per group)

// c[t][v] = C(v + t, t + 1): the colex-rank term of value v at position t
// (at most C(67, 4) = 766480).
struct SymTab {
    int32_t c[SYM_T][SYM_V];
};

// Tile::pad0 of a tile in this mode: SYM_TILE | parent tie pattern << 8 | u_0 << 16
// (pattern bit t: u_t = u_{t+1}); Tile::pad1 = canonical rows of the parent.
constexpr int32_t SYM_TILE = 2;
STTSM_HD bool sym_tile(int32_t pad0) { return (pad0 & 3) == SYM_TILE; }
STTSM_HD uint32_t sym_pattern(int32_t pad0) { return ((uint32_t)pad0 >> 8) & 0xff; }
STTSM_HD int sym_u0(int32_t pad0) { return (int)((uint32_t)pad0 >> 16); }

// Table entries i, i + stride, ... (one thread per i on the device; 0, 1 on the
// host): C(v + t, t + 1) = prod_{i=1}^{t+1} (v - 1 + i) / i, each partial product
// an integer below 2^23.
STTSM_HD void sym_tab_fill(SymTab& T, int i0, int stride)
{
    for (int i = i0; i < SYM_T * SYM_V; i += stride) {
        const int t = i / SYM_V, v = i - t * SYM_V;
        int32_t c = 1;
        for (int j = 1; j <= t + 1; ++j) c = c * (v - 1 + j) / j;
        T.c[t][v] = c;
    }
}

// Largest v < vlim with ct[v] <= r (ct[0] = 0, ct increasing in v; vlim <= 64).
STTSM_HD int sym_find(const int32_t* ct, int32_t r, int vlim)
{
    int lo = 0;
#pragma unroll
    for (int step = 32; step > 0; step >>= 1)
        if (lo + step < vlim && ct[lo + step] <= r) lo += step;
    return lo;
}

// Non-decreasing tuple s_0 <= ... <= s_{len-1} over [0, vlim) of colex rank r,
// packed 8 bits per value (s_t at bits 8t); len <= SYM_T.
STTSM_HD uint32_t sym_unrank(const SymTab& T, int32_t r, int len, int vlim)
{
    uint32_t out = 0;
#pragma unroll
    for (int t = SYM_T - 1; t >= 0; --t) {
        if (t < len) {
            const int v = sym_find(T.c[t], r, vlim);
            out |= (uint32_t)v << (8 * t);
            r -= T.c[t][v];
        }
    }
    return out;
}

// Number of canonical rows of a parent with the given tie pattern at level k.
STTSM_HD int64_t sym_parent_rows(const SymTab& T, int m, int k, int b, int Kp, uint32_t pattern)
{
    const int d = m - 1 - k;
    int64_t rows = k == 0 ? 1 : (int64_t)T.c[k - 1][Kp];
    for (int t = 0; t < d;) {
        int g = 1;
        while (t + g < d && ((pattern >> (t + g - 1)) & 1)) ++g;
        rows *= T.c[g - 1][b];
        t += g;
    }
    return rows;
}

// Canonical row rho of a parent: returns its row pr * R + rr among the
// parent's rows (the row map of the full computation) and, in *tie, bit a
// set where modes a and a + 1 (both != k) hold the same block; *iblk gets the
// i blocks I_0 <= ... <= I_{k-1}, 8 bits each (I_t < nbar <= 64).  The parent's
// canonical rows number less than 2^31 (they are at most its rows), so the
// rank arithmetic is 32-bit; tuples stay packed in registers.
STTSM_HD int64_t sym_row(const SymTab& T, int m, int k, int b, int Kp, int64_t R, const int32_t* bpow, uint32_t pattern,
                         int64_t rho, uint32_t* tie, uint32_t* iblk)
{
    const int d = m - 1 - k;
    int lb = -1;   // log2 b for a power of two
    if ((b & (b - 1)) == 0) {
        lb = 0;
        while ((1 << lb) < b) ++lb;
    }
    const uint32_t Ni = k == 0 ? 1u : (uint32_t)T.c[k - 1][Kp];
    uint32_t rj = (uint32_t)rho / Ni;
    const uint32_t ri = (uint32_t)rho - rj * Ni;
    int64_t pr = 0, rr = 0;
    uint32_t tb = 0, ib = 0;
    if (k > 0) {
        const uint32_t xs = sym_unrank(T, (int32_t)ri, k, Kp);
        int prev = -1;
#pragma unroll
        for (int t = 0; t < SYM_T; ++t) {
            if (t < k) {
                const int x = (int)((xs >> (8 * t)) & 0xff);
                const int blk = lb >= 0 ? x >> lb : x / b;
                pr += T.c[t][blk];
                rr += (int64_t)(x - blk * b) * bpow[t];
                ib |= (uint32_t)blk << (8 * t);
                if (t > 0 && blk == prev) tb |= 1u << (t - 1);
                prev = blk;
            }
        }
    }
    for (int t = 0; t < d;) {
        int g = 1;
        while (t + g < d && ((pattern >> (t + g - 1)) & 1)) ++g;
        const uint32_t cnt = (uint32_t)T.c[g - 1][b];
        const uint32_t q = rj / cnt;
        const uint32_t rk = rj - q * cnt;
        rj = q;
        const uint32_t ys = sym_unrank(T, (int32_t)rk, g, b);
        for (int u = 0; u < g; ++u) {
            rr += (int64_t)((ys >> (8 * u)) & 0xff) * bpow[k + t + u];   // mode k+1+t+u is row digit k+t+u
            if (u + 1 < g) tb |= 1u << (k + 1 + t + u);
        }
        t += g;
    }
    *tie = tb;
    *iblk = ib;
    return pr * R + rr;
}

// Next distinct permutation of o[lo .. hi) in lexicographic order; at the
// last one, restores the non-decreasing order and returns false.
STTSM_HD bool sym_next_perm(int32_t* o, int lo, int hi)
{
    int i = hi - 2;
    while (i >= lo && o[i] >= o[i + 1]) --i;
    if (i < lo) {
        for (int a = lo, z = hi - 1; a < z; ++a, --z) { const int32_t w = o[a]; o[a] = o[z]; o[z] = w; }
        return false;
    }
    int j = hi - 1;
    while (o[j] <= o[i]) --j;
    { const int32_t w = o[i]; o[i] = o[j]; o[j] = w; }
    for (int a = i + 1, z = hi - 1; a < z; ++a, --z) { const int32_t w = o[a]; o[a] = o[z]; o[z] = w; }
    return true;
}
