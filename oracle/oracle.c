/*
 * CPU correctness oracle for string sorting with LCP output.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  The CUDA library never calls
 * it and shares no code, header, table or helper with it.
 *
 * Plain, slow and written to be checked by eye against the paper
 * (Bingmann, Eberle, Sanders, "Engineering Parallel String Sorting"):
 *
 *   orc_sort            the problem of Section 2: sort n strings
 *                       lexicographically; ties between equal strings by
 *                       ascending input index; LCP array with lcp[0] = 0.
 *   orc_stats           L = sum of the LCP array and the distinguishing
 *                       prefix size D (Section 2), D by its closed form.
 *   orc_chars_h         chars_h(s): the 8 characters at depth h, big-endian,
 *                       zero past the end of the string (Section 4.4).
 *   orc_s5_tree         level-order splitter tree t from in-order splitters
 *                       x (Algorithm 1, tree construction; Figure 1).
 *   orc_s5_classify     classification of keys by descending t and one
 *                       equality test (Algorithm 1, classification loop).
 *   orc_s5_classify_equal  the S5-Equal alternative of Section 4.4: an
 *                       equality test at every node of one descent.
 *   orc_s5_distribute   bucket counts, prefix sum and stable out-of-place
 *                       redistribution (Algorithm 1, count / prefix sum /
 *                       redistribute).
 *   orc_s5_pick         splitter selection from a sorted sample with the
 *                       recursive "skip equal samples" scheme (Section 4.4).
 *   orc_lcp_insertion   LCP-aware insertion sort (Algorithm 5).
 *   orc_lcp_compare     LCP-Compare (Algorithm 2).
 *   orc_lcp_merge2      binary LCP-merge (Algorithm 3).
 *   orc_lcp_mergek      K-way LCP-merge with an LCP-aware loser tree
 *                       (Algorithm 4).
 *
 * String model: string i starts at chars[offsets[i]].  If lengths != NULL it
 * has lengths[i] bytes; else if fixed_len != 0 it has fixed_len bytes; else it
 * ends at the first 0 byte.  Characters are unsigned bytes 1..255 (the paper's
 * alphabet {1..sigma}); the end of a string compares below every character.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - equal strings are ordered by ascending input index;
 *   - perm[i] is the input index of the i-th smallest string;
 *   - lcp[0] = 0, the LCP with the empty string;
 *   - the LCP of two strings stops at the end of the shorter one;
 *   - splitter tree descent goes right when c > t_i, so the in-order leaf
 *     index is r = #{j : x_j < c} and the bucket is 2r + [r < v and x_r = c].
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const uint8_t *chars;
    const uint64_t *offsets;
    const uint32_t *lengths;
    uint32_t fixed_len;
} orc_set;

/* ---------------------------------------------------------------- strings */

static uint64_t str_len(const orc_set *S, uint64_t i)
{
    if (S->lengths) return S->lengths[i];
    if (S->fixed_len) return S->fixed_len;
    const uint8_t *p = S->chars + S->offsets[i];
    uint64_t k = 0;
    while (p[k] != 0) k++;
    return k;
}

/* character at position k (0-based) of string i; 0 at and past the end */
static unsigned str_at(const orc_set *S, uint64_t i, uint64_t k, uint64_t len)
{
    if (k >= len) return 0;
    return S->chars[S->offsets[i] + k];
}

/* lexicographic comparison, the end of a string below every character */
static int str_cmp(const orc_set *S, uint64_t a, uint64_t b)
{
    uint64_t la = str_len(S, a), lb = str_len(S, b);
    uint64_t m = la < lb ? la : lb;
    int c = memcmp(S->chars + S->offsets[a], S->chars + S->offsets[b], m);
    if (c != 0) return c < 0 ? -1 : 1;
    if (la == lb) return 0;
    return la < lb ? -1 : 1;
}

/* lcp(s_a, s_b): number of leading positions where both strings agree */
static uint64_t str_lcp(const orc_set *S, uint64_t a, uint64_t b)
{
    uint64_t la = str_len(S, a), lb = str_len(S, b);
    uint64_t m = la < lb ? la : lb;
    const uint8_t *pa = S->chars + S->offsets[a], *pb = S->chars + S->offsets[b];
    uint64_t k = 0;
    while (k < m && pa[k] == pb[k]) k++;
    return k;
}

static int cmp_index(const void *x, const void *y, void *ctx)
{
    const orc_set *S = (const orc_set *)ctx;
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    int c = str_cmp(S, a, b);
    if (c != 0) return c;
    return (a > b) - (a < b);   /* ties: ascending input index */
}

/* ------------------------------------------------------- sort (Section 2) */

int orc_sort(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
             uint32_t fixed_len, uint64_t n, uint32_t *perm, uint32_t *lcp)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    for (uint64_t i = 0; i < n; i++) perm[i] = (uint32_t)i;
    qsort_r(perm, n, sizeof(uint32_t), cmp_index, &S);
    if (lcp) {
        if (n) lcp[0] = 0;
        for (uint64_t i = 1; i < n; i++)
            lcp[i] = (uint32_t)str_lcp(&S, perm[i - 1], perm[i]);
    }
    return 0;
}

/* naive LCP array of a given order (used to check any claimed output) */
void orc_lcp_of(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                uint32_t fixed_len, uint64_t n, const uint32_t *perm, uint32_t *lcp)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    if (n) lcp[0] = 0;
    for (uint64_t i = 1; i < n; i++) lcp[i] = (uint32_t)str_lcp(&S, perm[i - 1], perm[i]);
}

/* sign of the comparison of strings a and b (-1, 0, +1) */
int orc_cmp(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
            uint32_t fixed_len, uint64_t a, uint64_t b)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    return str_cmp(&S, a, b);
}

/*
 * L and D of Section 2.  L = sum_{i>=1} lcp[i].  D counts, for every string,
 * the characters inspected to place it: its longest LCP with a sorted
 * neighbour plus the distinguishing character, at most the whole string plus
 * its terminator: dist_i = min(max(lcp[i], lcp[i+1]) + 1, |s_i| + 1), with
 * lcp[0] = lcp[n] = 0.  Also returns N = sum (|s_i| + 1).
 */
void orc_stats(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
               uint32_t fixed_len, uint64_t n, const uint32_t *perm, const uint32_t *lcp,
               uint64_t *L_out, uint64_t *D_out, uint64_t *N_out)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    uint64_t L = 0, D = 0, N = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t left = i ? lcp[i] : 0;
        uint64_t right = (i + 1 < n) ? lcp[i + 1] : 0;
        uint64_t m = (left > right ? left : right) + 1;
        uint64_t len = str_len(&S, perm[i]);
        D += m < len + 1 ? m : len + 1;
        N += len + 1;
        if (i) L += lcp[i];
    }
    *L_out = L;
    *D_out = D;
    *N_out = N;
}

/* -------------------------------------------- chars_h (Section 4.4, w = 8) */

uint64_t orc_chars_h(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                     uint32_t fixed_len, uint64_t i, uint64_t h)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    uint64_t len = str_len(&S, i);
    uint64_t key = 0;
    for (int k = 0; k < 8; k++)   /* first character in the most significant byte */
        key = (key << 8) | str_at(&S, i, h + (uint64_t)k, len);
    return key;
}

void orc_chars_h_all(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                     uint32_t fixed_len, uint64_t n, const uint64_t *depth, uint64_t *keys)
{
    for (uint64_t i = 0; i < n; i++)
        keys[i] = orc_chars_h(chars, offsets, lengths, fixed_len, i, depth[i]);
}

/* ----------------------------------------------- one S5 step (Algorithm 1) */

/*
 * Level-order tree t[1..v] (stored at t[0..v-1]) of the in-order splitters
 * x_0..x_{v-1}, v = 2^d - 1: the root is the middle splitter, then the middle
 * splitters of the two halves, and so on (Figure 1: v = 7 gives
 * x3, x1, x5, x0, x2, x4, x6).
 */
void orc_s5_tree(const uint64_t *x, uint32_t v, uint64_t *t)
{
    uint32_t vp = v + 1;   /* v' = v + 1 = 2^d */
    uint32_t node = 1;
    for (uint32_t step = vp; step >= 2; step /= 2) {
        /* this level holds x_{step/2 - 1}, x_{3 step/2 - 1}, ... */
        for (uint32_t j = step / 2; j < vp; j += step) t[node++ - 1] = x[j - 1];
    }
}

/*
 * Classify each key c: descend the level-order tree with i := 2i + [c > t_i]
 * for log2(v+1) levels, take the in-order leaf index r = i - (v + 1), and
 * test equality with x_r once.  Bucket 2r: x_{r-1} < c < x_r; bucket 2r+1:
 * c = x_r.  (x_v is the sentinel infinity, so r = v gives bucket 2v.)
 */
void orc_s5_classify(const uint64_t *keys, uint64_t n, const uint64_t *x, uint32_t v,
                     uint16_t *bucket)
{
    uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * (v ? v : 1));
    orc_s5_tree(x, v, t);
    uint32_t d = 0;
    while ((1u << d) < v + 1) d++;
    for (uint64_t j = 0; j < n; j++) {
        uint64_t c = keys[j];
        uint32_t i = 1;
        for (uint32_t lvl = 0; lvl < d; lvl++) i = 2 * i + (c > t[i - 1] ? 1 : 0);
        uint32_t r = i - (v + 1);
        uint32_t m = 2 * r;
        if (r < v && x[r] == c) m++;
        bucket[j] = (uint16_t)m;
    }
    free(t);
}

/*
 * S5-Equal (the fourth way of placing the equality test in Section 4.4): one
 * descent of t per key that tests c = t_i at every node and stops at the
 * first node that holds c.  Node i of level l (2^l <= i < 2^(l+1)) holds the
 * in-order splitter x_k with k = (2 (i - 2^l) + 1) 2^(d-l-1) - 1 (the inverse
 * of the level-order layout of Figure 1), so a stop there is bucket 2k + 1.
 * A descent that meets no equal splitter ends at leaf i of level d in the
 * even bucket 2 (i - 2^d).  With distinct splitters this is orc_s5_classify's
 * bucket; where a splitter value repeats, c stops at the copy nearest the
 * root on its path, an equality bucket of the same value.
 */
void orc_s5_classify_equal(const uint64_t *keys, uint64_t n, const uint64_t *x, uint32_t v,
                           uint16_t *bucket)
{
    uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * (v ? v : 1));
    orc_s5_tree(x, v, t);
    uint32_t d = 0;
    while ((1u << d) < v + 1) d++;
    for (uint64_t j = 0; j < n; j++) {
        uint64_t c = keys[j];
        uint32_t i = 1;
        int stopped = 0;
        uint32_t m = 0;
        for (uint32_t lvl = 0; lvl < d; lvl++) {
            if (c == t[i - 1]) {
                uint32_t k = ((2 * (i - (1u << lvl)) + 1) << (d - lvl - 1)) - 1;
                m = 2 * k + 1;
                stopped = 1;
                break;
            }
            i = 2 * i + (c > t[i - 1] ? 1 : 0);
        }
        if (!stopped) m = 2 * (i - (1u << d));
        bucket[j] = (uint16_t)m;
    }
    free(t);
}

/*
 * Counting, prefix sum and stable out-of-place redistribution of one step.
 * bucket_begin[b] = first output position of bucket b (2v+2 entries, the
 * last = n); out[p] = the input position placed at p.  Strings keep their
 * input order inside a bucket.
 */
void orc_s5_distribute(const uint16_t *bucket, uint64_t n, uint32_t v,
                       uint64_t *bucket_begin, uint64_t *out)
{
    uint32_t k = 2 * v + 1;
    uint64_t *cnt = (uint64_t *)calloc(k + 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) cnt[bucket[i]]++;
    uint64_t run = 0;
    for (uint32_t b = 0; b < k; b++) {
        bucket_begin[b] = run;
        run += cnt[b];
    }
    bucket_begin[k] = run;
    for (uint32_t b = 0; b < k; b++) cnt[b] = bucket_begin[b];
    for (uint64_t i = 0; i < n; i++) out[cnt[bucket[i]]++] = i;
    free(cnt);
}

/*
 * Splitter selection of Section 4.4 from a sorted sample p[0..a-1]: take the
 * middle sample of range [lo, hi) as the middle splitter of the current
 * subtree, skip the samples equal to it on both sides, recurse on the left
 * and right remainders.  An empty range repeats the nearest splitter on its
 * right (the bound of the subtree), or the one on its left at the right end,
 * so x stays sorted.  Writes v in-order splitters.
 */
static void pick_rec(const uint64_t *p, int64_t lo, int64_t hi, uint64_t *x, uint32_t xlo,
                     uint32_t xhi, int has_right, uint64_t right, uint64_t left)
{
    if (xlo >= xhi) return;
    uint32_t xm = xlo + (xhi - xlo) / 2;
    if (lo >= hi) {
        uint64_t fill = has_right ? right : left;
        for (uint32_t j = xlo; j < xhi; j++) x[j] = fill;
        return;
    }
    int64_t m = lo + (hi - lo) / 2;
    uint64_t s = p[m];
    int64_t b = m, a = m;
    while (b > lo && p[b - 1] == s) b--;
    while (a < hi && p[a] == s) a++;
    x[xm] = s;
    pick_rec(p, lo, b, x, xlo, xm, 1, s, left);
    pick_rec(p, a, hi, x, xm + 1, xhi, has_right, right, s);
}

void orc_s5_pick(const uint64_t *sorted_sample, uint64_t a, uint32_t v, uint64_t *x)
{
    pick_rec(sorted_sample, 0, (int64_t)a, x, 0, v, 0, 0, 0);
}

/* ------------------------------------------------- LCP-Compare (Alg. 2) */

/*
 * Strings s_a, s_b with h_a = lcp(p, s_a), h_b = lcp(p, s_b) for a common
 * predecessor p <= s_a, s_b.  Returns 0 when s_a comes first and 1 when s_b
 * comes first; *hp = lcp(s_a, s_b).  Case 1 (h_a = h_b) compares characters
 * from h_a on; case 2 (h_a < h_b) means s_b < s_a; case 3 (h_a > h_b) means
 * s_a < s_b.  Equal strings (both end at the same place) go to a unless
 * b_on_tie is set.  Every evaluation of the character loop condition counts
 * as one character comparison.
 */
static int lcp_compare(const orc_set *S, uint64_t sa, uint64_t ha, uint64_t sb, uint64_t hb,
                       int b_on_tie, uint64_t *hp, uint64_t *ncmp)
{
    if (ha == hb) {
        uint64_t la = str_len(S, sa), lb = str_len(S, sb);
        uint64_t h = ha;
        unsigned ca, cb;
        for (;;) {
            ca = str_at(S, sa, h, la);
            cb = str_at(S, sb, h, lb);
            (*ncmp)++;
            if (ca != 0 && ca == cb) { h++; continue; }
            break;
        }
        *hp = h;
        if (ca < cb) return 0;
        if (ca > cb) return 1;
        return b_on_tie ? 1 : 0;
    }
    if (ha < hb) { *hp = ha; return 1; }
    *hp = hb;
    return 0;
}

/* out = {x, h_x, y, h'}: winner string, its LCP to p, loser string, lcp(s_a, s_b) */
uint64_t orc_lcp_compare(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                         uint32_t fixed_len, uint64_t a, uint64_t ha, uint64_t b, uint64_t hb,
                         uint64_t *out)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    uint64_t ncmp = 0, hp = 0;
    int r = lcp_compare(&S, a, ha, b, hb, 0, &hp, &ncmp);
    out[0] = r ? b : a;
    out[1] = r ? hb : ha;
    out[2] = r ? a : b;
    out[3] = hp;
    return ncmp;
}

/* -------------------------------------------- binary LCP-merge (Alg. 3) */

/*
 * Merge sorted runs s1[0..n1) and s2[0..n2) (string indices) with LCP arrays
 * h1, h2 (entry 0 unused) into out/hout.  Invariant: hk = lcp of run k's
 * front string with the last string written.  After writing the smaller
 * front s_x, run x advances and takes its stored LCP, the other run takes
 * lcp(s_1, s_2) from LCP-Compare.  An exhausted run is the sentinel infinity.
 * Equal strings: run 1 first.  Returns the number of character comparisons.
 */
uint64_t orc_lcp_merge2(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                        uint32_t fixed_len, const uint32_t *s1, const uint32_t *h1, uint64_t n1,
                        const uint32_t *s2, const uint32_t *h2, uint64_t n2, uint32_t *out,
                        uint32_t *hout)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    uint64_t i1 = 0, i2 = 0, j = 0, ncmp = 0;
    uint64_t hk1 = 0, hk2 = 0;
    while (i1 < n1 || i2 < n2) {
        int both = (i1 < n1) && (i2 < n2);
        uint64_t hp = 0;
        int take2 = both ? lcp_compare(&S, s1[i1], hk1, s2[i2], hk2, 0, &hp, &ncmp) : (i1 >= n1);
        if (!take2) {
            out[j] = s1[i1];
            hout[j] = (uint32_t)hk1;
            j++;
            i1++;
            hk1 = (i1 < n1) ? h1[i1] : 0;
            if (both) hk2 = hp;
        } else {
            out[j] = s2[i2];
            hout[j] = (uint32_t)hk2;
            j++;
            i2++;
            hk2 = (i2 < n2) ? h2[i2] : 0;
            if (both) hk1 = hp;
        }
    }
    if (j) hout[0] = 0;
    return ncmp;
}

/* -------------------------------------------- K-way LCP-merge (Alg. 4) */

/*
 * K sorted runs given as concatenated string indices s[] and LCP arrays h[],
 * run k occupying [begin[k], begin[k+1]).  Loser tree over K' = 2^ceil(log2 K)
 * inputs, one-based: input k is leaf K' + k, internal node i (1..K'-1) holds
 * (loser input y_i, h_i = LCP of that loser with the winner of the game at
 * i); the overall winner w and its LCP h_w to the last output are kept
 * apart.  The initial games are all played bottom-up with every LCP equal
 * to the common prefix 0.  After writing s_w, input w advances, takes its
 * stored LCP to s_w, and replays the games on its leaf-to-root path; each
 * stored h_i is then an LCP with s_w, the common predecessor LCP-Compare
 * needs.  Exhausted inputs are the sentinel infinity.  Equal strings go to
 * the lower input number.  Returns the number of character comparisons.
 */
typedef struct {
    const orc_set *S;
    const uint32_t *s;
    const uint64_t *end;
    const uint64_t *pos;
    uint64_t *ncmp;
} kctx;

/* one game of inputs a and b; LCPs ha, hb to the common predecessor */
static void kgame(kctx *C, uint64_t a, uint64_t ha, uint64_t b, uint64_t hb,
                  uint64_t *x, uint64_t *hx, uint64_t *y, uint64_t *hy)
{
    int ea = C->pos[a] >= C->end[a], eb = C->pos[b] >= C->end[b];
    int bwins;
    uint64_t hp = 0;
    if (ea || eb) bwins = (ea && !eb) || (ea && eb && b < a);
    else bwins = lcp_compare(C->S, C->s[C->pos[a]], ha, C->s[C->pos[b]], hb, b < a, &hp, C->ncmp);
    if (bwins) { *x = b; *hx = hb; *y = a; }
    else       { *x = a; *hx = ha; *y = b; }
    *hy = hp;
}

uint64_t orc_lcp_mergek(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                        uint32_t fixed_len, const uint32_t *s, const uint32_t *h,
                        const uint64_t *begin, uint32_t K, uint32_t *out, uint32_t *hout)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    uint32_t Kp = 1;
    while (Kp < K) Kp *= 2;
    uint64_t *pos = (uint64_t *)calloc(Kp, sizeof(uint64_t));
    uint64_t *end = (uint64_t *)calloc(Kp, sizeof(uint64_t));
    uint64_t *yv = (uint64_t *)calloc(2 * Kp, sizeof(uint64_t));
    uint64_t *hv = (uint64_t *)calloc(2 * Kp, sizeof(uint64_t));
    uint64_t ncmp = 0, total = 0;
    for (uint32_t k = 0; k < Kp; k++) {
        pos[k] = k < K ? begin[k] : 0;
        end[k] = k < K ? begin[k + 1] : 0;
        if (k < K) total += end[k] - pos[k];
    }
    kctx C = {&S, s, end, pos, &ncmp};
    uint64_t w = 0, hw = 0;
    if (Kp > 1) {
        /* initial games, bottom-up: wv[i] = winner below node i */
        uint64_t *wv = (uint64_t *)calloc(2 * Kp, sizeof(uint64_t));
        for (uint32_t k = 0; k < Kp; k++) wv[Kp + k] = k;
        for (uint32_t i = Kp - 1; i >= 1; i--) {
            uint64_t x, hx, y, hy;
            kgame(&C, wv[2 * i], 0, wv[2 * i + 1], 0, &x, &hx, &y, &hy);
            wv[i] = x;
            yv[i] = y;
            hv[i] = hy;
        }
        w = wv[1];
        free(wv);
    }
    for (uint64_t j = 0; j < total; j++) {
        out[j] = s[pos[w]];
        hout[j] = (uint32_t)(j ? hw : 0);
        ((uint64_t *)pos)[w]++;
        uint64_t x = w, hx = (pos[w] < end[w]) ? h[pos[w]] : 0;
        for (uint32_t node = (Kp + (uint32_t)w) / 2; node >= 1; node /= 2) {
            uint64_t nx, nhx, ny, nhy;
            kgame(&C, x, hx, yv[node], hv[node], &nx, &nhx, &ny, &nhy);
            x = nx;
            hx = nhx;
            yv[node] = ny;
            hv[node] = nhy;
        }
        w = x;
        hw = hx;
    }
    free(pos);
    free(end);
    free(yv);
    free(hv);
    return ncmp;
}

/* ---------------------------------------- LCP insertion sort (Alg. 5) */

/*
 * Sort the strings s[0..n) that share a common prefix of hbar characters, in
 * place, and write their LCP array to h[0..n) (h[0] = 0).  One-based arrays
 * A[1..n] and H[1..n+1] follow the paper's notation: when x = s_j is
 * inserted, the hole moves left from position j; H[i] is then the LCP of the
 * strings left and right of the hole and h' the LCP of x with the string
 * right of the hole (hbar at the start).  H[i] < h': x goes here.  H[i] = h':
 * compare characters from h'.  H[i] > h': shift without comparing.  Equal
 * strings keep their given order.  Returns the number of evaluations of the
 * character loop condition.
 */
uint64_t orc_lcp_insertion(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                           uint32_t fixed_len, uint32_t *s, uint32_t *h, uint64_t n, uint64_t hbar)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    uint64_t ncmp = 0;
    uint32_t *A = (uint32_t *)malloc(sizeof(uint32_t) * (n + 1));
    uint64_t *H = (uint64_t *)calloc(n + 2, sizeof(uint64_t));
    for (uint64_t k = 1; k <= n; k++) A[k] = s[k - 1];
    for (uint64_t j = 1; j <= n; j++) {
        uint64_t i = j;
        uint32_t x = A[j];
        uint64_t hp = hbar;
        uint64_t lx = str_len(&S, x);
        while (i > 1) {
            if (H[i] < hp) break;
            if (H[i] == hp) {
                uint64_t p = hp;
                uint32_t left = A[i - 1];
                uint64_t ll = str_len(&S, left);
                for (;;) {
                    unsigned cx = str_at(&S, x, hp, lx), cl = str_at(&S, left, hp, ll);
                    ncmp++;
                    if (cx != 0 && cx == cl) { hp++; continue; }
                    break;
                }
                if (str_at(&S, x, hp, lx) >= str_at(&S, left, hp, ll)) {
                    H[i] = hp;
                    hp = p;
                    break;
                }
            }
            A[i] = A[i - 1];
            H[i + 1] = H[i];
            i--;
        }
        A[i] = x;
        H[i + 1] = hp;
    }
    for (uint64_t k = 1; k <= n; k++) {
        s[k - 1] = A[k];
        h[k - 1] = (uint32_t)(k >= 2 ? H[k] : 0);
    }
    free(A);
    free(H);
    return ncmp;
}

/* ------------------------------------------- checks of a claimed output */

/*
 * Check a claimed sorted order and LCP array against the definitions of
 * Section 2 at every position: perm is a permutation of 0..n-1, each
 * neighbouring pair is in order (equal strings by ascending index), lcp[0]
 * = 0 and lcp[i] is the naive LCP of the neighbours.  Returns the number of
 * failing positions; *first gets the first one (or n when none fails).
 */
uint64_t orc_check_sorted(const uint8_t *chars, const uint64_t *offsets, const uint32_t *lengths,
                          uint32_t fixed_len, uint64_t n, const uint32_t *perm, const uint32_t *lcp,
                          uint64_t *first)
{
    orc_set S = {chars, offsets, lengths, fixed_len};
    uint64_t bad = 0;
    *first = n;
    uint8_t *seen = (uint8_t *)calloc(n ? n : 1, 1);
    for (uint64_t i = 0; i < n; i++) {
        int ok = perm[i] < n && !seen[perm[i]];
        if (perm[i] < n) seen[perm[i]] = 1;
        if (ok && i == 0) ok = lcp[0] == 0;
        if (ok && i > 0 && perm[i - 1] < n) {
            int c = str_cmp(&S, perm[i - 1], perm[i]);
            ok = c < 0 || (c == 0 && perm[i - 1] < perm[i]);
            if (ok) ok = lcp[i] == str_lcp(&S, perm[i - 1], perm[i]);
        }
        if (!ok) {
            if (*first == n) *first = i;
            bad++;
        }
    }
    free(seen);
    return bad;
}
