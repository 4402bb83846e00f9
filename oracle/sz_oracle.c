/*
 * sz_oracle.c -- plain, slow, single-threaded CPU oracle for the SZ-LV path of
 * "In-Depth Exploration of Single-Snapshot Lossy Compression Techniques for
 * N-Body Simulations" (Tao, Di, Chen, Cappello; arXiv 1711.03888).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path; the stream layout it writes is
 * restated here from the format description, independently of the kernels.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared sz_oracle.c -lm
 * Floating point: IEEE binary64 '/', '*', '-', nearbyint() in the default
 * round-to-nearest-even mode, and the (float) conversion (round to nearest).
 *
 * What each function follows (paper sections / tables / equations):
 *   error bound ......... Sec. III "Pointwise compression error": e_i < eb_abs,
 *                         eb_rel = eb_abs / R with R = max - min.
 *   lattice ............. Sec. II (CPC2000 step 1: floats become integers by
 *                         dividing by the error bound); the lattice step is
 *                         2*eb so the rounding error stays within eb.
 *   prediction .......... Sec. IV-A, last-value (LV) model: pred_i = x_{i-1},
 *                         applied on the integer lattice; and the original
 *                         SZ's linear-curve-fitting (LCF) model,
 *                         pred_i = 2 x_{i-1} - x_{i-2}, on the same lattice.
 *   quantization ........ Sec. IV-A: linear-scaling quantization with a very
 *                         large number of intervals (2^16 here, radius 32768);
 *                         values outside are stored aside (escapes).
 *   Huffman ............. Sec. II / IV-B: Huffman coding of the quantization
 *                         codes (two-queue construction, canonical codes).
 *   R-index ............. Sec. IV-B, Fig. 3(a): bit-interleave of the integer
 *                         coordinates; segment-wise radix sort (Table 4) that
 *                         ignores the lowest p 3-bit digits (Table 5).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <float.h>

/* ---- stream layout constants (restated from the format description) ---- */
#define O_MAGIC        0x564C5A53u   /* 'S','Z','L','V' little-endian */
#define O_VERSION      1u
#define O_HEADER_BYTES 160u
#define O_MAX_LEN      24            /* longest Huffman codeword, bits */
#define O_M_BITS       16            /* 2^16 quantization codes */
#define O_RADIUS       32768         /* code = delta + radius; code 0 = escape */
#define O_FLAG_RAW        1u
#define O_FLAG_REORDERED  2u
#define O_ESC_BYTES    16u
#define O_PRED_LV      1u            /* header byte 43: predictor */
#define O_PRED_LCF     2u

/* return codes (mirrors the meaning of the C-ABI status values) */
#define SZO_OK       0
#define SZO_ERR_ARG  1
#define SZO_ERR_NOMEM 2
#define SZO_ERR_CAPACITY 3
#define SZO_ERR_CORRUPT 4

static uint64_t pad16(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

static void put_u16(uint8_t* p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t* p, uint32_t v) { for (int k = 0; k < 4; ++k) p[k] = (uint8_t)(v >> (8 * k)); }
static void put_u64(uint8_t* p, uint64_t v) { for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(v >> (8 * k)); }
static uint16_t get_u16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t get_u32(const uint8_t* p) { uint32_t v = 0; for (int k = 3; k >= 0; --k) v = (v << 8) | p[k]; return v; }
static uint64_t get_u64(const uint8_t* p) { uint64_t v = 0; for (int k = 7; k >= 0; --k) v = (v << 8) | p[k]; return v; }
static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint64_t d2u(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
static double u2d(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }

/* ------------------------------------------------------------------------ */
/* Sec. III: value range over the finite values and the absolute error bound */
/* ------------------------------------------------------------------------ */

/* R = max - min over the finite elements (0 when there are none). */
double szo_value_range(const float* x, uint64_t n)
{
    int any = 0;
    float lo = 0.0f, hi = 0.0f;
    for (uint64_t i = 0; i < n; ++i) {
        if (!isfinite(x[i])) continue;
        if (!any) { lo = hi = x[i]; any = 1; continue; }
        if (x[i] < lo) lo = x[i];
        if (x[i] > hi) hi = x[i];
    }
    if (!any) return 0.0;
    return (double)hi - (double)lo;
}

/* Lattice step: the largest float not above 2*eb_abs (clamped to FLT_MAX). */
float szo_step(double eb_abs)
{
    double two = 2.0 * eb_abs;
    if (two >= (double)FLT_MAX) return FLT_MAX;
    float f = (float)two;
    if ((double)f > two) f = nextafterf(f, 0.0f);
    return f;
}

/* eb given as absolute (kind 0) or value-range relative (kind 1). */
int szo_error_bound(const float* x, uint64_t n, double eb, int kind, double* eb_abs, float* step)
{
    if (!(eb >= 0.0) || !isfinite(eb) || (kind != 0 && kind != 1)) return SZO_ERR_ARG;
    double e = (kind == 1) ? eb * szo_value_range(x, n) : eb;
    if (!isfinite(e)) return SZO_ERR_ARG;
    *eb_abs = e;
    *step = szo_step(e);
    return SZO_OK;
}

/* ------------------------------------------------------------------------ */
/* Value -> lattice, and the reconstruction check that decides "verbatim"    */
/* ------------------------------------------------------------------------ */

static void lattice_one(float x, float D, double eb_abs, int64_t* q, int* verbatim)
{
    if (!isfinite(x)) { *q = 0; *verbatim = 1; return; }
    double t = (double)x / (double)D;
    if (!(fabs(t) < 9007199254740992.0)) { *q = 0; *verbatim = 1; return; }   /* 2^53 */
    int64_t k = (int64_t)nearbyint(t);
    float xr = (float)((double)k * (double)D);
    *q = k;
    *verbatim = fabs((double)x - (double)xr) > eb_abs;
}

void szo_lattice(const float* x, uint64_t n, float D, double eb_abs, int64_t* q, uint8_t* verbatim)
{
    for (uint64_t i = 0; i < n; ++i) {
        int v;
        lattice_one(x[i], D, eb_abs, &q[i], &v);
        verbatim[i] = (uint8_t)v;
    }
}

/* Lattice -> value (decoder side). */
float szo_recon(int64_t q, float D) { return (float)((double)q * (double)D); }

/* LV prediction on the lattice + linear-scaling quantization (Sec. IV-A).
 * code[i] = delta + 32768 for |delta| <= 32767 and not verbatim, else 0. */
void szo_codes(const int64_t* q, const uint8_t* verbatim, uint64_t n, uint16_t* code, int64_t* delta)
{
    int64_t prev = 0;
    for (uint64_t i = 0; i < n; ++i) {
        int64_t d = q[i] - prev;
        delta[i] = d;
        if (verbatim[i] || d < -(O_RADIUS - 1) || d > (O_RADIUS - 1)) code[i] = 0;
        else code[i] = (uint16_t)(d + O_RADIUS);
        prev = q[i];
    }
}

/* LCF prediction on the lattice (Sec. IV-A, the original SZ's linear curve
 * fitting: pred_i = 2 x_{i-1} - x_{i-2}), with q_{-1} = q_{-2} = 0:
 * delta_i = q_i - 2 q_{i-1} + q_{i-2}; codes as for LV. */
void szo_codes_lcf(const int64_t* q, const uint8_t* verbatim, uint64_t n, uint16_t* code, int64_t* delta)
{
    int64_t p1 = 0, p2 = 0;
    for (uint64_t i = 0; i < n; ++i) {
        int64_t d = q[i] - 2 * p1 + p2;
        delta[i] = d;
        if (verbatim[i] || d < -(O_RADIUS - 1) || d > (O_RADIUS - 1)) code[i] = 0;
        else code[i] = (uint16_t)(d + O_RADIUS);
        p2 = p1;
        p1 = q[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Huffman code lengths: two-queue construction, then canonical codes       */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t f; uint32_t sym; uint32_t k; } leaf_t;

static int leaf_cmp(const void* a, const void* b)
{
    const leaf_t* x = (const leaf_t*)a;
    const leaf_t* y = (const leaf_t*)b;
    if (x->f != y->f) return x->f < y->f ? -1 : 1;
    return x->sym < y->sym ? -1 : (x->sym > y->sym ? 1 : 0);
}

/* m used symbols, given in ascending symbol order with their frequencies.
 * Leaves are ordered by (frequency, symbol); at equal weights a leaf is taken
 * before an internal node, and internal nodes are taken in creation order.
 * A leaf's length is its depth.  If the deepest leaf exceeds 24 bits every
 * frequency f becomes (f >> 1) | 1 and the construction is repeated. */
int szo_huffman_lengths(const uint64_t* freq, const uint32_t* sym, uint32_t m, uint8_t* len)
{
    if (m == 0) return SZO_OK;
    if (m == 1) { len[0] = 1; return SZO_OK; }
    uint64_t* f = (uint64_t*)malloc(sizeof(uint64_t) * m);
    leaf_t* lv = (leaf_t*)malloc(sizeof(leaf_t) * m);
    uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * (2 * (size_t)m - 1));
    uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * (2 * (size_t)m - 1));
    uint32_t* depth = (uint32_t*)malloc(sizeof(uint32_t) * (2 * (size_t)m - 1));
    if (!f || !lv || !w || !parent || !depth) {
        free(f); free(lv); free(w); free(parent); free(depth);
        return SZO_ERR_NOMEM;
    }
    for (uint32_t k = 0; k < m; ++k) f[k] = freq[k];
    for (;;) {
        for (uint32_t k = 0; k < m; ++k) { lv[k].f = f[k]; lv[k].sym = sym[k]; lv[k].k = k; }
        qsort(lv, m, sizeof(leaf_t), leaf_cmp);
        /* node ids: 0..m-1 leaves in sorted order, m..2m-2 internal in creation order */
        for (uint32_t k = 0; k < m; ++k) w[k] = lv[k].f;
        uint32_t lf = 0, ifr = m, iend = m;
        while (iend < 2 * m - 1) {
            uint32_t pick[2];
            for (int t = 0; t < 2; ++t) {
                if (lf < m && (ifr == iend || w[lf] <= w[ifr])) pick[t] = lf++;
                else pick[t] = ifr++;
            }
            w[iend] = w[pick[0]] + w[pick[1]];
            parent[pick[0]] = iend;
            parent[pick[1]] = iend;
            ++iend;
        }
        uint32_t root = 2 * m - 2;
        depth[root] = 0;
        for (int64_t v = (int64_t)root - 1; v >= 0; --v) depth[v] = depth[parent[v]] + 1;
        uint32_t maxd = 0;
        for (uint32_t k = 0; k < m; ++k) if (depth[k] > maxd) maxd = depth[k];
        if (maxd <= O_MAX_LEN) {
            for (uint32_t k = 0; k < m; ++k) len[lv[k].k] = (uint8_t)depth[k];
            break;
        }
        for (uint32_t k = 0; k < m; ++k) f[k] = (f[k] >> 1) | 1u;
    }
    free(f); free(lv); free(w); free(parent); free(depth);
    return SZO_OK;
}

/* Canonical codewords: ordered by (length, symbol); the first code of each
 * length is (first code of the previous length + its count) shifted left. */
void szo_canonical_codes(const uint8_t* len, uint32_t m, uint32_t* code)
{
    uint32_t count[O_MAX_LEN + 2] = {0};
    uint32_t next[O_MAX_LEN + 2] = {0};
    for (uint32_t k = 0; k < m; ++k) count[len[k]]++;
    uint32_t c = 0;
    count[0] = 0;
    for (int l = 1; l <= O_MAX_LEN; ++l) {
        c = (c + count[l - 1]) << 1;
        next[l] = c;
    }
    for (uint32_t k = 0; k < m; ++k) code[k] = next[len[k]]++;   /* symbols ascending */
}

/* ------------------------------------------------------------------------ */
/* Stream writer                                                            */
/* ------------------------------------------------------------------------ */

uint64_t szo_max_bytes(uint64_t n)
{
    return O_HEADER_BYTES + 4u * ((n + 3u) & ~(uint64_t)3u);
}

static int valid_params(uint64_t n, uint32_t C, uint32_t G)
{
    if (n >= ((uint64_t)1 << 32)) return 0;
    if (C < 256 || C > 65536 || (C & (C - 1))) return 0;
    if (G < 16 || G > 2048 || (G & (G - 1)) || G > C) return 0;
    return 1;
}

static void put_bits(uint8_t* payload, uint64_t* bitpos, uint32_t cw, int len)
{
    /* payload is a little-endian u32 word array; bit 31 of word 0 comes first */
    for (int b = len - 1; b >= 0; --b) {
        if ((cw >> b) & 1u) {
            uint64_t word = *bitpos >> 5;
            uint32_t bit = 31u - (uint32_t)(*bitpos & 31u);
            payload[4 * word + bit / 8] |= (uint8_t)(1u << (bit % 8));
        }
        (*bitpos)++;
    }
}

static void write_header(uint8_t* out, uint64_t n, double eb_abs, float D, uint32_t flags,
                         uint32_t C, uint32_t G, uint32_t pred, uint64_t n_chunks, uint64_t n_sym,
                         uint64_t n_esc, uint64_t payload_words, const uint64_t off[8], uint64_t total)
{
    memset(out, 0, O_HEADER_BYTES);
    put_u32(out + 0, O_MAGIC);
    put_u16(out + 4, (uint16_t)O_VERSION);
    put_u16(out + 6, (uint16_t)O_HEADER_BYTES);
    put_u64(out + 8, n);
    put_u64(out + 16, d2u(eb_abs));
    put_u32(out + 24, f2u(D));
    put_u32(out + 28, flags);
    put_u32(out + 32, C);
    put_u32(out + 36, G);
    put_u16(out + 40, (uint16_t)O_M_BITS);
    out[42] = (uint8_t)O_MAX_LEN;
    out[43] = (uint8_t)pred;           /* predictor: 1 last value, 2 linear curve fitting */
    put_u64(out + 48, n_chunks);
    put_u64(out + 56, n_sym);
    put_u64(out + 64, n_esc);
    put_u64(out + 72, payload_words);
    for (int s = 0; s < 8; ++s) put_u64(out + 80 + 8 * s, off[s]);
    put_u64(out + 144, total);
}

static int write_raw(const float* x, uint64_t n, double eb_abs, float D, uint32_t flags,
                     uint32_t C, uint32_t G, uint32_t pred, uint8_t* out, uint64_t cap, uint64_t* out_bytes)
{
    uint64_t words = (n + 3u) & ~(uint64_t)3u;
    uint64_t total = O_HEADER_BYTES + 4u * words;
    *out_bytes = total;
    if (cap < total) return SZO_ERR_CAPACITY;
    uint64_t off[8];
    for (int s = 0; s < 8; ++s) off[s] = O_HEADER_BYTES;
    write_header(out, n, eb_abs, D, flags | O_FLAG_RAW, C, G, pred, 0, 0, 0, words, off, total);
    memset(out + O_HEADER_BYTES, 0, 4u * words);
    for (uint64_t i = 0; i < n; ++i) put_u32(out + O_HEADER_BYTES + 4 * i, f2u(x[i]));
    return SZO_OK;
}

/* Compress one float32 array.  kind: 0 = absolute eb, 1 = value-range relative.
 * C = elements per chunk, G = elements per sub-stream (powers of two).
 * extra_flags: O_FLAG_REORDERED when the caller reordered the array.
 * pred: O_PRED_LV or O_PRED_LCF (the LCF chunk anchors are q_{b-1}, q_{b-2}). */
int szo_compress_pred(const float* x, uint64_t n, double eb, int kind, uint32_t C, uint32_t G,
                      uint32_t extra_flags, uint32_t pred, uint8_t* out, uint64_t cap, uint64_t* out_bytes)
{
    *out_bytes = 0;
    if (!valid_params(n, C, G) || (pred != O_PRED_LV && pred != O_PRED_LCF)) return SZO_ERR_ARG;
    double eb_abs; float D;
    int rc = szo_error_bound(x, n, eb, kind, &eb_abs, &D);
    if (rc) return rc;
    uint32_t flags = extra_flags & O_FLAG_REORDERED;
    if (n == 0) {
        uint64_t off[8];
        for (int s = 0; s < 8; ++s) off[s] = O_HEADER_BYTES;
        *out_bytes = O_HEADER_BYTES;
        if (cap < O_HEADER_BYTES) return SZO_ERR_CAPACITY;
        write_header(out, 0, eb_abs, D, flags, C, G, pred, 0, 0, 0, 0, off, O_HEADER_BYTES);
        return SZO_OK;
    }
    if (D == 0.0f) return write_raw(x, n, eb_abs, D, flags, C, G, pred, out, cap, out_bytes);

    int64_t* q = (int64_t*)malloc(8 * n);
    int64_t* delta = (int64_t*)malloc(8 * n);
    uint8_t* verb = (uint8_t*)malloc(n);
    uint16_t* code = (uint16_t*)malloc(2 * n);
    uint64_t* hist = (uint64_t*)calloc(65536, sizeof(uint64_t));
    if (!q || !delta || !verb || !code || !hist) {
        free(q); free(delta); free(verb); free(code); free(hist);
        return SZO_ERR_NOMEM;
    }
    szo_lattice(x, n, D, eb_abs, q, verb);
    if (pred == O_PRED_LCF) szo_codes_lcf(q, verb, n, code, delta);
    else szo_codes(q, verb, n, code, delta);
    uint64_t n_esc = 0;
    for (uint64_t i = 0; i < n; ++i) { hist[code[i]]++; if (code[i] == 0) n_esc++; }

    /* codebook over the used symbols, ascending */
    uint32_t m = 0;
    for (uint32_t s = 0; s < 65536; ++s) if (hist[s]) m++;
    uint32_t* sym = (uint32_t*)malloc(4 * (size_t)m);
    uint64_t* fr = (uint64_t*)malloc(8 * (size_t)m);
    uint8_t* len = (uint8_t*)malloc(m);
    uint32_t* cw = (uint32_t*)malloc(4 * (size_t)m);
    uint32_t* sym_len = (uint32_t*)calloc(65536, 4);
    uint32_t* sym_cw = (uint32_t*)calloc(65536, 4);
    if (!sym || !fr || !len || !cw || !sym_len || !sym_cw) { rc = SZO_ERR_NOMEM; goto done; }
    m = 0;
    for (uint32_t s = 0; s < 65536; ++s) if (hist[s]) { sym[m] = s; fr[m] = hist[s]; m++; }
    rc = szo_huffman_lengths(fr, sym, m, len);
    if (rc) goto done;
    szo_canonical_codes(len, m, cw);
    uint64_t B = 0;
    for (uint32_t k = 0; k < m; ++k) {
        sym_len[sym[k]] = len[k];
        sym_cw[sym[k]] = cw[k];
        B += fr[k] * len[k];
    }

    /* section layout */
    uint64_t n_chunks = (n + C - 1) / C;
    uint64_t S = C / G;
    uint64_t off[8];
    uint64_t o = O_HEADER_BYTES;
    off[0] = o; o = pad16(o + 2 * (uint64_t)m);              /* symbols u16 */
    off[1] = o; o = pad16(o + (uint64_t)m);                  /* lengths u8 */
    off[2] = o; o = pad16(o + 8 * (n_chunks + 1));           /* chunk word offsets u64 */
    const uint64_t n_anchor = pred == O_PRED_LCF ? 2 : 1;
    off[3] = o; o = pad16(o + 8 * n_anchor * n_chunks);      /* chunk anchors i64 (LCF: two each) */
    off[4] = o; o = pad16(o + 8 * (n_chunks + 1));           /* chunk escape bases u64 */
    off[5] = o; o = pad16(o + 2 * n_chunks * S);             /* sub-stream bit lengths u16 */
    off[6] = o; o = pad16(o + (uint64_t)O_ESC_BYTES * n_esc); /* escape records */
    off[7] = o;                                              /* payload u32 words */

    uint64_t raw_total = O_HEADER_BYTES + 4u * ((n + 3u) & ~(uint64_t)3u);
    uint64_t bound = off[7] + (B + 128u * n_chunks + 7u) / 8u;
    if (bound >= raw_total) {
        rc = write_raw(x, n, eb_abs, D, flags, C, G, pred, out, cap, out_bytes);
        goto done;
    }

    /* payload size: every chunk padded to a multiple of 128 bits */
    uint64_t words = 0;
    for (uint64_t c = 0; c < n_chunks; ++c) {
        uint64_t bits = 0;
        uint64_t e = (c + 1) * C < n ? (c + 1) * C : n;
        for (uint64_t i = c * C; i < e; ++i) bits += sym_len[code[i]];
        words += 4 * ((bits + 127) / 128);
    }
    uint64_t total = off[7] + 4 * words;
    *out_bytes = total;
    if (cap < total) { rc = SZO_ERR_CAPACITY; goto done; }
    memset(out, 0, total);
    write_header(out, n, eb_abs, D, flags, C, G, pred, n_chunks, m, n_esc, words, off, total);
    for (uint32_t k = 0; k < m; ++k) {
        put_u16(out + off[0] + 2 * k, (uint16_t)sym[k]);
        out[off[1] + k] = len[k];
    }
    {
        uint8_t* payload = out + off[7];
        uint64_t wpos = 0, esc = 0;
        for (uint64_t c = 0; c < n_chunks; ++c) {
            uint64_t b0 = c * C;
            uint64_t e = b0 + C < n ? b0 + C : n;
            put_u64(out + off[2] + 8 * c, wpos);
            put_u64(out + off[3] + 8 * n_anchor * c, (uint64_t)(b0 >= 1 ? q[b0 - 1] : 0));
            if (pred == O_PRED_LCF) put_u64(out + off[3] + 8 * (2 * c + 1), (uint64_t)(b0 >= 2 ? q[b0 - 2] : 0));
            put_u64(out + off[4] + 8 * c, esc);
            uint64_t bitpos = 32 * wpos;
            for (uint64_t k = 0; k < S; ++k) {
                uint64_t s0 = b0 + k * G;
                uint64_t s1 = s0 + G < e ? s0 + G : e;
                uint64_t start = bitpos;
                for (uint64_t i = s0; i < s1; ++i) {
                    put_bits(payload, &bitpos, sym_cw[code[i]], (int)sym_len[code[i]]);
                    if (code[i] == 0) {
                        uint8_t* r = out + off[6] + O_ESC_BYTES * esc;
                        put_u64(r, (uint64_t)delta[i]);
                        put_u32(r + 8, verb[i] ? f2u(x[i]) : 0u);
                        put_u32(r + 12, verb[i] ? 1u : 0u);
                        esc++;
                    }
                }
                put_u16(out + off[5] + 2 * (c * S + k), (uint16_t)(s0 < e ? bitpos - start : 0));
            }
            wpos += 4 * ((bitpos - 32 * wpos + 127) / 128);
        }
        put_u64(out + off[2] + 8 * n_chunks, wpos);
        put_u64(out + off[4] + 8 * n_chunks, esc);
    }
    rc = SZO_OK;
done:
    free(q); free(delta); free(verb); free(code); free(hist);
    free(sym); free(fr); free(len); free(cw); free(sym_len); free(sym_cw);
    return rc;
}

int szo_compress(const float* x, uint64_t n, double eb, int kind, uint32_t C, uint32_t G,
                 uint32_t extra_flags, uint8_t* out, uint64_t cap, uint64_t* out_bytes)
{
    return szo_compress_pred(x, n, eb, kind, C, G, extra_flags, O_PRED_LV, out, cap, out_bytes);
}

/* ------------------------------------------------------------------------ */
/* Stream reader                                                            */
/* ------------------------------------------------------------------------ */

static int get_bit(const uint8_t* payload, uint64_t bitpos)
{
    uint64_t word = bitpos >> 5;
    uint32_t bit = 31u - (uint32_t)(bitpos & 31u);
    return (payload[4 * word + bit / 8] >> (bit % 8)) & 1;
}

/* Returns the element count of a stream (header only), or an error. */
int szo_stream_n(const uint8_t* in, uint64_t in_bytes, uint64_t* n)
{
    if (in_bytes < O_HEADER_BYTES || get_u32(in) != O_MAGIC || get_u16(in + 4) != O_VERSION)
        return SZO_ERR_CORRUPT;
    *n = get_u64(in + 8);
    return SZO_OK;
}

int szo_decompress(const uint8_t* in, uint64_t in_bytes, float* out, uint64_t n_cap, uint64_t* n_out)
{
    *n_out = 0;
    uint64_t n;
    if (szo_stream_n(in, in_bytes, &n)) return SZO_ERR_CORRUPT;
    float D = u2f(get_u32(in + 24));
    uint32_t flags = get_u32(in + 28);
    uint32_t C = get_u32(in + 32), G = get_u32(in + 36);
    uint64_t n_chunks = get_u64(in + 48), m = get_u64(in + 56), n_esc = get_u64(in + 64);
    uint64_t words = get_u64(in + 72), total = get_u64(in + 144);
    uint32_t pred = in[43];
    uint64_t off[8];
    for (int s = 0; s < 8; ++s) off[s] = get_u64(in + 80 + 8 * s);
    if (total > in_bytes || off[7] + 4 * words > total || !valid_params(n, C, G)) return SZO_ERR_CORRUPT;
    if (pred != O_PRED_LV && pred != O_PRED_LCF) return SZO_ERR_CORRUPT;
    *n_out = n;
    if (n > n_cap) return SZO_ERR_CAPACITY;
    if (n == 0) return SZO_OK;
    if (flags & O_FLAG_RAW) {
        if (4 * n > 4 * words) return SZO_ERR_CORRUPT;
        for (uint64_t i = 0; i < n; ++i) out[i] = u2f(get_u32(in + off[7] + 4 * i));
        return SZO_OK;
    }
    if (n_chunks != (n + C - 1) / C || m == 0 || m > 65536) return SZO_ERR_CORRUPT;
    uint64_t S = C / G;
    if (off[6] + O_ESC_BYTES * n_esc > off[7] || off[5] + 2 * n_chunks * S > off[6]) return SZO_ERR_CORRUPT;
    if (off[2] + 8 * (n_chunks + 1) > off[3] || off[3] + 8 * (pred == O_PRED_LCF ? 2 : 1) * n_chunks > off[4] ||
        off[4] + 8 * (n_chunks + 1) > off[5])
        return SZO_ERR_CORRUPT;

    /* canonical decode tables: count per length, first code, symbols by (len, sym) */
    uint32_t count[O_MAX_LEN + 2] = {0}, first[O_MAX_LEN + 2] = {0}, base[O_MAX_LEN + 2] = {0};
    uint32_t* by_len = (uint32_t*)malloc(4 * m);
    if (!by_len) return SZO_ERR_NOMEM;
    for (uint64_t k = 0; k < m; ++k) {
        uint32_t l = in[off[1] + k];
        if (l < 1 || l > O_MAX_LEN) { free(by_len); return SZO_ERR_CORRUPT; }
        count[l]++;
    }
    {
        uint32_t c = 0, b = 0;
        for (int l = 1; l <= O_MAX_LEN; ++l) {
            c = (c + count[l - 1]) << 1;
            first[l] = c;
            base[l] = b;
            b += count[l];
        }
        uint32_t fill[O_MAX_LEN + 2];
        memcpy(fill, base, sizeof(fill));
        for (uint64_t k = 0; k < m; ++k) by_len[fill[in[off[1] + k]]++] = get_u16(in + off[0] + 2 * k);
    }
    const uint8_t* payload = in + off[7];
    int rc = SZO_OK;
    for (uint64_t c = 0; c < n_chunks && rc == SZO_OK; ++c) {
        uint64_t b0 = c * C;
        uint64_t e = b0 + C < n ? b0 + C : n;
        uint64_t wpos = get_u64(in + off[2] + 8 * c);
        uint64_t wend = get_u64(in + off[2] + 8 * (c + 1));
        /* LV: q_i = q_{i-1} + delta_i.  LCF: q_i = 2 q_{i-1} - q_{i-2} + delta_i
         * (two's-complement wrap on corrupt input) */
        const uint64_t n_anchor = pred == O_PRED_LCF ? 2 : 1;
        int64_t qv = (int64_t)get_u64(in + off[3] + 8 * n_anchor * c);
        int64_t qv2 = pred == O_PRED_LCF ? (int64_t)get_u64(in + off[3] + 8 * (2 * c + 1)) : 0;
        uint64_t esc = get_u64(in + off[4] + 8 * c);
        if (wend > words || wpos > wend) { rc = SZO_ERR_CORRUPT; break; }
        uint64_t bitpos = 32 * wpos;
        for (uint64_t k = 0; k < S && rc == SZO_OK; ++k) {
            uint64_t s0 = b0 + k * G;
            uint64_t s1 = s0 + G < e ? s0 + G : e;
            for (uint64_t i = s0; i < s1; ++i) {
                uint32_t cv = 0, sv = 0;
                int found = 0;
                for (int l = 1; l <= O_MAX_LEN; ++l) {
                    if (bitpos >= 32 * wend) { rc = SZO_ERR_CORRUPT; break; }
                    cv = (cv << 1) | (uint32_t)get_bit(payload, bitpos++);
                    if (count[l] && cv - first[l] < count[l]) { sv = by_len[base[l] + cv - first[l]]; found = 1; break; }
                }
                if (!found) { rc = SZO_ERR_CORRUPT; break; }
                int64_t d;
                int verbatim = 0;
                uint32_t raw = 0;
                if (sv == 0) {
                    if (esc >= n_esc) { rc = SZO_ERR_CORRUPT; break; }
                    const uint8_t* r = in + off[6] + O_ESC_BYTES * esc;
                    d = (int64_t)get_u64(r);
                    raw = get_u32(r + 8);
                    verbatim = (int)(get_u32(r + 12) & 1u);
                    esc++;
                } else {
                    d = (int64_t)sv - O_RADIUS;
                }
                if (pred == O_PRED_LCF) {
                    int64_t qn = (int64_t)(2 * (uint64_t)qv - (uint64_t)qv2 + (uint64_t)d);
                    qv2 = qv;
                    qv = qn;
                } else {
                    qv = (int64_t)((uint64_t)qv + (uint64_t)d);
                }
                out[i] = verbatim ? u2f(raw) : szo_recon(qv, D);
            }
        }
    }
    free(by_len);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* MD reordering: R-index (Fig. 3a) and segment-wise partial radix sort     */
/* ------------------------------------------------------------------------ */

/* Interleave three integers: bit 3k+2 = x_k, bit 3k+1 = y_k, bit 3k = z_k. */
uint64_t szo_morton3(uint64_t ux, uint64_t uy, uint64_t uz, int b)
{
    uint64_t key = 0;
    for (int k = 0; k < b; ++k) {
        key |= ((ux >> k) & 1u) << (3 * k + 2);
        key |= ((uy >> k) & 1u) << (3 * k + 1);
        key |= ((uz >> k) & 1u) << (3 * k);
    }
    return key;
}

/* R-index keys of n particles from their lattice coordinates:
 * u = q - min(q) per axis; b = bit length of the largest u (at most 21 kept:
 * the lowest bits are dropped so that 3b <= 63). */
void szo_rindex_keys(const int64_t* qx, const int64_t* qy, const int64_t* qz, uint64_t n, uint64_t* key, int* bits_out)
{
    if (n == 0) { *bits_out = 0; return; }
    const int64_t* q[3] = {qx, qy, qz};
    int64_t qmin[3];
    uint64_t umax = 0;
    for (int a = 0; a < 3; ++a) {
        qmin[a] = q[a][0];
        for (uint64_t i = 1; i < n; ++i) if (q[a][i] < qmin[a]) qmin[a] = q[a][i];
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t u = (uint64_t)(q[a][i] - qmin[a]);
            if (u > umax) umax = u;
        }
    }
    int b = 0;
    while (b < 64 && (umax >> b) != 0) ++b;
    int drop = b > 21 ? b - 21 : 0;
    if (b > 21) b = 21;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t u[3];
        for (int a = 0; a < 3; ++a) u[a] = (uint64_t)(q[a][i] - qmin[a]) >> drop;
        key[i] = szo_morton3(u[0], u[1], u[2], b);
    }
    *bits_out = b;
}

typedef struct { uint64_t k; uint64_t i; } ki_t;

static int ki_cmp(const void* a, const void* b)
{
    const ki_t* x = (const ki_t*)a;
    const ki_t* y = (const ki_t*)b;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    return x->i < y->i ? -1 : (x->i > y->i ? 1 : 0);
}

/* Stable sort of each segment of S elements by key >> 3p (Table 5: p ignored
 * 3-bit digits).  perm[j] = original index of the element placed at j. */
int szo_segment_sort(const uint64_t* key, uint64_t n, uint32_t S, uint32_t p, uint32_t* perm)
{
    if (S == 0 || p > 21) return SZO_ERR_ARG;
    ki_t* buf = (ki_t*)malloc(sizeof(ki_t) * (S ? S : 1));
    if (!buf) return SZO_ERR_NOMEM;
    for (uint64_t s0 = 0; s0 < n; s0 += S) {
        uint64_t e = s0 + S < n ? s0 + S : n;
        for (uint64_t i = s0; i < e; ++i) { buf[i - s0].k = key[i] >> (3 * p); buf[i - s0].i = i; }
        qsort(buf, e - s0, sizeof(ki_t), ki_cmp);   /* (key, index): a stable order */
        for (uint64_t i = s0; i < e; ++i) perm[i] = (uint32_t)buf[i - s0].i;
    }
    free(buf);
    return SZO_OK;
}

/* Full MD reordering for a snapshot: lattice coordinates of fields 0..2 with
 * their own steps, keys, segment sort.  Writes perm (n entries). */
int szo_rindex_perm(const float* x, const float* y, const float* z, uint64_t n,
                    const float D[3], const double eb_abs[3], uint32_t S, uint32_t p,
                    uint32_t* perm, uint64_t* key_out)
{
    int64_t* q[3];
    uint8_t* v = (uint8_t*)malloc(n ? n : 1);
    uint64_t* key = (uint64_t*)malloc(8 * (n ? n : 1));
    const float* f[3] = {x, y, z};
    int rc = SZO_OK;
    for (int a = 0; a < 3; ++a) q[a] = (int64_t*)malloc(8 * (n ? n : 1));
    if (!v || !key || !q[0] || !q[1] || !q[2]) { rc = SZO_ERR_NOMEM; goto out; }
    for (int a = 0; a < 3; ++a) {
        if (D[a] == 0.0f) { for (uint64_t i = 0; i < n; ++i) q[a][i] = 0; continue; }
        szo_lattice(f[a], n, D[a], eb_abs[a], q[a], v);
    }
    int b;
    szo_rindex_keys(q[0], q[1], q[2], n, key, &b);
    rc = szo_segment_sort(key, n, S, p, perm);
    if (key_out) memcpy(key_out, key, 8 * n);
out:
    free(v); free(key); free(q[0]); free(q[1]); free(q[2]);
    return rc;
}

/* Snapshot compression in the LV_PRX mode: the first three fields are the
 * coordinates; every field is reordered by the same permutation (no index
 * array is stored, Sec. IV-B) and compressed with LV.  out[f] must hold
 * szo_max_bytes(n) bytes. */
int szo_compress_snapshot(int nfields, const float* const* in, uint64_t n, const double* eb, int kind,
                          uint32_t C, uint32_t G, uint32_t S, uint32_t p,
                          uint8_t* const* out, const uint64_t* cap, uint64_t* out_bytes, uint32_t* perm_out)
{
    if (nfields < 3) return SZO_ERR_ARG;
    double ea[3]; float D[3];
    for (int a = 0; a < 3; ++a) {
        int rc = szo_error_bound(in[a], n, eb[a], kind, &ea[a], &D[a]);
        if (rc) return rc;
    }
    uint32_t* perm = (uint32_t*)malloc(4 * (n ? n : 1));
    float* tmp = (float*)malloc(4 * (n ? n : 1));
    if (!perm || !tmp) { free(perm); free(tmp); return SZO_ERR_NOMEM; }
    int rc = szo_rindex_perm(in[0], in[1], in[2], n, D, ea, S, p, perm, NULL);
    for (int f = 0; f < nfields && rc == SZO_OK; ++f) {
        for (uint64_t j = 0; j < n; ++j) tmp[j] = in[f][perm[j]];
        rc = szo_compress(tmp, n, eb[f], kind, C, G, O_FLAG_REORDERED, out[f], cap[f], &out_bytes[f]);
    }
    if (perm_out && rc == SZO_OK) memcpy(perm_out, perm, 4 * n);
    free(perm); free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* SZ-CPC2000 coordinates (Sec. II CPC2000 steps 1-4; Sec. IV-B SZ-CPC2000)  */
/* ------------------------------------------------------------------------ */
/*
 * Step 1: each coordinate onto its own lattice (the SZ-LV lattice and
 * verbatim rule).  Step 2: the lossless R-index key of every particle (bit
 * 3k+2 = x_k, 3k+1 = y_k, 3k = z_k of u = q - min q; 3b <= 63 or the bound
 * is too fine for the key).  Step 3: all particles stably sorted by key and
 * the differences of adjacent keys taken.  Step 4: the differences coded
 * with a Rice code whose parameter k is chosen per block of 4096 particles
 * (the paper's "adaptive variable-length code" is not given; this is the
 * reading): d >> k zero bits, a one bit, then the low k bits of d, MSB-first.
 * Each block restarts from its first key (stored raw), so blocks decode
 * independently; 32 sub-streams of 128 particles per block carry their bit
 * offsets.  Verbatim coordinates are exception records.
 *
 * Stream ("SZCP", version 1, little-endian), sections on 16-byte boundaries:
 *   0 u32 magic 0x50435A53 | 4 u16 version | 6 u16 header bytes (160)
 *   8 u64 n | 16 f64 eb_abs[3] | 40 u32 D[3] (float bits) | 52 u32 b
 *   56 i64 qmin[3] | 80 u32 block (4096) | 84 u32 sub-streams per block (32)
 *   88 u64 n_blocks | 96 u64 n_exceptions | 104 u64 payload words
 *   112 u64 offsets: first keys u64[nb] | 120 block word offsets u64[nb+1]
 *   128 Rice parameters u8[nb] | 136 sub-stream bit offsets u32[nb*32]
 *   144 exceptions {u64 position, u32 axis, u32 raw bits}[ne] | 152 payload
 */
#define O_CPC_MAGIC   0x50435A53u
#define O_CPC_BLOCK   4096u
#define O_CPC_SUBS    32u
#define O_CPC_SUBLEN  (O_CPC_BLOCK / O_CPC_SUBS)
#define SZO_ERR_UNSUPPORTED 5

uint64_t szo_cpc_rice_bits(uint64_t d, int k) { return (d >> k) + 1u + (uint64_t)k; }

/* k in [0, 63] minimising the Rice bits of d[0..L) (the smallest on ties) */
int szo_cpc_choose_k(const uint64_t* d, uint64_t L)
{
    int best_k = 0;
    uint64_t best = UINT64_MAX;
    for (int k = 0; k < 64; ++k) {
        uint64_t t = 0;
        for (uint64_t i = 0; i < L; ++i) t += szo_cpc_rice_bits(d[i], k);
        if (t < best) { best = t; best_k = k; }
    }
    return best_k;
}

static void put_bits64(uint8_t* payload, uint64_t* bitpos, uint64_t v, int len)
{
    for (int i = len - 1; i >= 0; --i) {
        if ((v >> i) & 1u) {
            uint64_t word = *bitpos >> 5;
            uint32_t bit = 31u - (uint32_t)(*bitpos & 31u);
            payload[4 * word + bit / 8] |= (uint8_t)(1u << (bit % 8));
        }
        (*bitpos)++;
    }
}

/* max(1, ...) allocations */
static void* zalloc(size_t b) { return calloc(b ? b : 1, 1); }

int szo_cpc_max_bytes(uint64_t n, uint64_t* bytes)
{
    uint64_t nb = (n + O_CPC_BLOCK - 1) / O_CPC_BLOCK;
    /* header + tables + 3 exceptions per particle + 65 bits per particle + padding */
    *bytes = O_HEADER_BYTES + 16 * 6 + 8 * nb + 8 * (nb + 1) + nb + 4 * O_CPC_SUBS * nb + 48 * n + 9 * n + 4 * nb + 64;
    return SZO_OK;
}

int szo_compress_cpc(const float* x, const float* y, const float* z, uint64_t n, const double eb[3], int kind,
                     uint8_t* out, uint64_t cap, uint64_t* out_bytes, uint32_t* perm_out)
{
    *out_bytes = 0;
    const float* f[3] = {x, y, z};
    double ea[3];
    float D[3];
    for (int a = 0; a < 3; ++a) {
        int rc = szo_error_bound(f[a], n, eb[a], kind, &ea[a], &D[a]);
        if (rc) return rc;
    }
    int64_t* q[3] = {NULL, NULL, NULL};
    uint8_t* vb[3] = {NULL, NULL, NULL};
    uint64_t* key = (uint64_t*)zalloc(8 * n);
    ki_t* kv = (ki_t*)zalloc(sizeof(ki_t) * n);
    uint64_t* d = (uint64_t*)zalloc(8 * O_CPC_BLOCK);
    int rc = SZO_OK;
    for (int a = 0; a < 3; ++a) { q[a] = (int64_t*)zalloc(8 * n); vb[a] = (uint8_t*)zalloc(n); }
    if (!key || !kv || !d || !q[0] || !q[1] || !q[2] || !vb[0] || !vb[1] || !vb[2]) { rc = SZO_ERR_NOMEM; goto out; }
    /* step 1 */
    for (int a = 0; a < 3; ++a) szo_lattice(f[a], n, D[a], ea[a], q[a], vb[a]);
    int64_t qmin[3] = {0, 0, 0};
    uint64_t umax = 0;
    for (int a = 0; a < 3 && n; ++a) {
        qmin[a] = q[a][0];
        for (uint64_t i = 1; i < n; ++i) if (q[a][i] < qmin[a]) qmin[a] = q[a][i];
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t u = (uint64_t)(q[a][i] - qmin[a]);
            if (u > umax) umax = u;
        }
    }
    int b = 0;
    while (b < 64 && (umax >> b) != 0) ++b;
    if (b > 21) { rc = SZO_ERR_UNSUPPORTED; goto out; }
    /* step 2 */
    for (uint64_t i = 0; i < n; ++i)
        key[i] = szo_morton3((uint64_t)(q[0][i] - qmin[0]), (uint64_t)(q[1][i] - qmin[1]),
                             (uint64_t)(q[2][i] - qmin[2]), b);
    /* step 3: stable sort by key */
    for (uint64_t i = 0; i < n; ++i) { kv[i].k = key[i]; kv[i].i = i; }
    qsort(kv, n, sizeof(ki_t), ki_cmp);
    /* layout */
    uint64_t nb = (n + O_CPC_BLOCK - 1) / O_CPC_BLOCK;
    uint64_t ne = 0;
    for (uint64_t j = 0; j < n; ++j)
        for (int a = 0; a < 3; ++a) ne += vb[a][kv[j].i];
    uint8_t* ks = (uint8_t*)zalloc(nb);
    uint64_t* bwords = (uint64_t*)zalloc(8 * (nb + 1));
    uint32_t* subs = (uint32_t*)zalloc(4 * O_CPC_SUBS * nb);
    if (!ks || !bwords || !subs) { free(ks); free(bwords); free(subs); rc = SZO_ERR_NOMEM; goto out; }
    uint64_t words = 0;
    for (uint64_t blk = 0; blk < nb; ++blk) {
        uint64_t j0 = blk * O_CPC_BLOCK, L = n - j0 < O_CPC_BLOCK ? n - j0 : O_CPC_BLOCK;
        for (uint64_t i = 0; i < L; ++i) d[i] = i ? kv[j0 + i].k - kv[j0 + i - 1].k : 0;
        int k = szo_cpc_choose_k(d, L);
        ks[blk] = (uint8_t)k;
        uint64_t bits = 0;
        for (uint32_t s = 0; s < O_CPC_SUBS; ++s) {
            subs[blk * O_CPC_SUBS + s] = (uint32_t)bits;
            for (uint64_t i = (uint64_t)s * O_CPC_SUBLEN; i < (uint64_t)(s + 1) * O_CPC_SUBLEN && i < L; ++i)
                bits += szo_cpc_rice_bits(d[i], k);
        }
        bwords[blk] = words;
        words += (bits + 31) / 32;
    }
    bwords[nb] = words;
    uint64_t off[6], o = O_HEADER_BYTES;
    off[0] = o; o = pad16(o + 8 * nb);
    off[1] = o; o = pad16(o + 8 * (nb + 1));
    off[2] = o; o = pad16(o + nb);
    off[3] = o; o = pad16(o + 4 * O_CPC_SUBS * nb);
    off[4] = o; o = pad16(o + 16 * ne);
    off[5] = o;
    uint64_t total = o + 4 * words;
    *out_bytes = total;
    if (cap < total) { rc = SZO_ERR_CAPACITY; free(ks); free(bwords); free(subs); goto out; }
    memset(out, 0, total);
    put_u32(out + 0, O_CPC_MAGIC);
    put_u16(out + 4, 1);
    put_u16(out + 6, (uint16_t)O_HEADER_BYTES);
    put_u64(out + 8, n);
    for (int a = 0; a < 3; ++a) {
        put_u64(out + 16 + 8 * a, d2u(ea[a]));
        put_u32(out + 40 + 4 * a, f2u(D[a]));
        put_u64(out + 56 + 8 * a, (uint64_t)qmin[a]);
    }
    put_u32(out + 52, (uint32_t)b);
    put_u32(out + 80, O_CPC_BLOCK);
    put_u32(out + 84, O_CPC_SUBS);
    put_u64(out + 88, nb);
    put_u64(out + 96, ne);
    put_u64(out + 104, words);
    for (int s = 0; s < 6; ++s) put_u64(out + 112 + 8 * s, off[s]);
    for (uint64_t blk = 0; blk < nb; ++blk) {
        uint64_t j0 = blk * O_CPC_BLOCK, L = n - j0 < O_CPC_BLOCK ? n - j0 : O_CPC_BLOCK;
        put_u64(out + off[0] + 8 * blk, kv[j0].k);
        out[off[2] + blk] = ks[blk];
        for (uint32_t s = 0; s < O_CPC_SUBS; ++s) put_u32(out + off[3] + 4 * (blk * O_CPC_SUBS + s), subs[blk * O_CPC_SUBS + s]);
        uint64_t bitpos = 32 * bwords[blk];
        for (uint64_t i = 0; i < L; ++i) {
            uint64_t dd = i ? kv[j0 + i].k - kv[j0 + i - 1].k : 0;
            int k = ks[blk];
            bitpos += dd >> k;                       /* zero bits */
            put_bits64(out + off[5], &bitpos, 1u, 1);
            if (k) put_bits64(out + off[5], &bitpos, dd & ((k == 64) ? ~0ull : ((1ull << k) - 1)), k);
        }
    }
    for (uint64_t blk = 0; blk <= nb; ++blk) put_u64(out + off[1] + 8 * blk, bwords[blk]);
    {
        uint64_t e = 0;
        for (uint64_t j = 0; j < n; ++j)
            for (int a = 0; a < 3; ++a)
                if (vb[a][kv[j].i]) {
                    uint8_t* r = out + off[4] + 16 * e++;
                    put_u64(r, j);
                    put_u32(r + 8, (uint32_t)a);
                    put_u32(r + 12, f2u(f[a][kv[j].i]));
                }
    }
    if (perm_out) for (uint64_t j = 0; j < n; ++j) perm_out[j] = (uint32_t)kv[j].i;
    free(ks); free(bwords); free(subs);
out:
    free(key); free(kv); free(d);
    for (int a = 0; a < 3; ++a) { free(q[a]); free(vb[a]); }
    return rc;
}

/* Inverse of the Morton interleave: u_axis from key (axis 0 = x leads). */
static uint64_t demorton(uint64_t key, int axis, int b)
{
    uint64_t u = 0;
    for (int k = 0; k < b; ++k) u |= ((key >> (3 * k + (2 - axis))) & 1u) << k;
    return u;
}

/* Decode an SZCP stream into the sorted coordinates (x, y, z hold n_cap). */
int szo_decompress_cpc(const uint8_t* in, uint64_t in_bytes, float* x, float* y, float* z, uint64_t n_cap,
                       uint64_t* n_out)
{
    *n_out = 0;
    if (in_bytes < O_HEADER_BYTES || get_u32(in) != O_CPC_MAGIC || get_u16(in + 4) != 1) return SZO_ERR_CORRUPT;
    uint64_t n = get_u64(in + 8), nb = get_u64(in + 88), ne = get_u64(in + 96), words = get_u64(in + 104);
    int b = (int)get_u32(in + 52);
    if (get_u32(in + 80) != O_CPC_BLOCK || get_u32(in + 84) != O_CPC_SUBS || b > 21) return SZO_ERR_CORRUPT;
    if (nb != (n + O_CPC_BLOCK - 1) / O_CPC_BLOCK) return SZO_ERR_CORRUPT;
    float D[3];
    int64_t qmin[3];
    uint64_t off[6];
    for (int a = 0; a < 3; ++a) { D[a] = u2f(get_u32(in + 40 + 4 * a)); qmin[a] = (int64_t)get_u64(in + 56 + 8 * a); }
    for (int s = 0; s < 6; ++s) off[s] = get_u64(in + 112 + 8 * s);
    if (off[0] < O_HEADER_BYTES || off[0] + 8 * nb > off[1] || off[1] + 8 * (nb + 1) > off[2] || off[2] + nb > off[3] ||
        off[3] + 4 * O_CPC_SUBS * nb > off[4] || off[4] + 16 * ne > off[5] || off[5] + 4 * words > in_bytes)
        return SZO_ERR_CORRUPT;
    *n_out = n;
    if (n > n_cap) return SZO_ERR_CAPACITY;
    float* o[3] = {x, y, z};
    const uint8_t* payload = in + off[5];
    for (uint64_t blk = 0; blk < nb; ++blk) {
        uint64_t j0 = blk * O_CPC_BLOCK, L = n - j0 < O_CPC_BLOCK ? n - j0 : O_CPC_BLOCK;
        uint64_t key = get_u64(in + off[0] + 8 * blk);
        uint64_t wb = get_u64(in + off[1] + 8 * blk), we = get_u64(in + off[1] + 8 * (blk + 1));
        int k = in[off[2] + blk];
        if (wb > we || we > words || k > 63) return SZO_ERR_CORRUPT;
        uint64_t bitpos = 32 * wb, end = 32 * we;
        for (uint64_t i = 0; i < L; ++i) {
            uint64_t zeros = 0;
            while (1) {
                if (bitpos >= end) return SZO_ERR_CORRUPT;
                if (get_bit(payload, bitpos++)) break;
                zeros++;
            }
            uint64_t r = 0;
            for (int t = 0; t < k; ++t) {
                if (bitpos >= end) return SZO_ERR_CORRUPT;
                r = (r << 1) | (uint64_t)get_bit(payload, bitpos++);
            }
            uint64_t dd = (zeros << k) | r;
            if (i) key += dd;
            for (int a = 0; a < 3; ++a) {
                int64_t qa = (int64_t)demorton(key, a, b) + qmin[a];
                o[a][j0 + i] = szo_recon(qa, D[a]);
            }
        }
    }
    for (uint64_t e = 0; e < ne; ++e) {
        const uint8_t* r = in + off[4] + 16 * e;
        uint64_t j = get_u64(r);
        uint32_t a = get_u32(r + 8);
        if (j >= n || a > 2) return SZO_ERR_CORRUPT;
        o[a][j] = u2f(get_u32(r + 12));
    }
    return SZO_OK;
}

/* ------------------------------------------------------------------------ */
/* R-index from coordinates and velocities (Sec. IV-C, Fig. 3b, Table 6)     */
/* ------------------------------------------------------------------------ */

/* Interleave six integers, one bit of each per 6-bit group, axis 0 leading:
 * bit 6k + (5 - a) = bit k of u[a]. */
uint64_t szo_morton6(const uint64_t u[6], int b)
{
    uint64_t key = 0;
    for (int k = 0; k < b; ++k)
        for (int a = 0; a < 6; ++a) key |= ((u[a] >> k) & 1u) << (6 * k + (5 - a));
    return key;
}

/* Keys of n particles from six lattice arrays (xx, yy, zz, vx, vy, vz):
 * u = q - min(q) per axis; b = bit length of the largest u, at most 10 kept
 * (the lowest bits dropped so that 6b <= 60). */
void szo_rindex_keys6(const int64_t* const* q, uint64_t n, uint64_t* key, int* bits_out)
{
    if (n == 0) { *bits_out = 0; return; }
    int64_t qmin[6];
    uint64_t umax = 0;
    for (int a = 0; a < 6; ++a) {
        qmin[a] = q[a][0];
        for (uint64_t i = 1; i < n; ++i) if (q[a][i] < qmin[a]) qmin[a] = q[a][i];
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t u = (uint64_t)(q[a][i] - qmin[a]);
            if (u > umax) umax = u;
        }
    }
    int b = 0;
    while (b < 64 && (umax >> b) != 0) ++b;
    int drop = b > 10 ? b - 10 : 0;
    if (b > 10) b = 10;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t u[6];
        for (int a = 0; a < 6; ++a) u[a] = (uint64_t)(q[a][i] - qmin[a]) >> drop;
        key[i] = szo_morton6(u, b);
    }
    *bits_out = b;
}
