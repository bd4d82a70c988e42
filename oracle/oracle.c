/*
 * oracle.c -- plain, slow, obviously-correct CPU definition of the tumour
 * database query of Ezhov et al., "A for-loop is all you need" (2022).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The CUDA library never
 * links it, and it shares no code, header or table with the CUDA path.
 *
 * What it computes (the paper's Section 2.3, "Query to a database of
 * synthetic tumors", and the "Baseline for-loop search" paragraph):
 *
 *   * each database volume u is thresholded at u_T1Gd and u_FLAIR, giving two
 *     binary segmentations per entry;  a voxel is in the mask when
 *     (float)u(x) >= t  (reading: ">=" compared in binary32);
 *   * each entry is compared with the patient's two segmentations by the
 *     Dice coefficient  Dice(A,B) = 2|A n B| / (|A| + |B|);  both masks
 *     empty counts as identical (Dice = 1);
 *   * the two Dice values are added and the entry with the largest sum is
 *     the best match; the score reported here is the mean
 *     (Dice_T1Gd + Dice_FLAIR) / 2, which orders entries identically because
 *     the halving is exact in binary64;
 *   * entries are ranked by (score descending, index ascending) -- the lowest
 *     index wins a tie -- and the first k are returned.
 *
 * Everything is a loop over voxels and entries, in the order the definition
 * states.  Counts are exact unsigned integers; the score is IEEE binary64,
 * round-to-nearest:  D_k = (double)(2 I_k) / (double)(P_k + E_k),
 * S = (D_1 + D_2) * 0.5.
 *
 * The half-precision storage path is decoded by this file's own IEEE
 * binary16 decoder (sign, 5-bit exponent with bias 15, 10-bit fraction,
 * subnormals, infinities, NaN), never by a library conversion.
 *
 * The embedding prefilter (low-dimensional retrieval, Section 2.3 "Autoencoders"
 * and "naive downsampling": L2 between compressed representations, combined as
 * L2_T1Gd + L2_FLAIR, lowest wins) is defined here as the f x f x f block mean
 * of each binary mask and the Euclidean distance between those block means,
 * computed in binary64.
 *
 * The prefilter's stored encodings are written out from their formats:
 * bfloat16 is binary32 rounded to nearest-even at bit 16; FP8 E4M3 (bias 7,
 * 3 fraction bits, largest finite 448, no infinity) is round-to-nearest-even
 * with saturation at +-448, applied to e / s with the per-row scale
 * s = max(e) / 448 computed in binary32 (s = 1 for an all-zero row).  The
 * decisions that produce those codes are taken in binary32, as the kernels
 * take them.
 *
 * The random-projection prefilter uses a count sketch of each binary mask
 * (a sparse random projection with one +-1 per voxel): voxel x goes to
 * bucket h(x) mod D with sign s(x), where h is the SplitMix64 output
 * function (Steele, Lea & Flood 2014) applied to (x + 1) * golden-ratio
 * increment; the sketch's squared L2 between two masks is an unbiased
 * estimate of the size of their symmetric difference.  The Hamming-code
 * prefilter keeps the sign bit [v > 0] of every bucket (a sign random
 * projection, the popcount analogue of the paper's hashing baseline) and
 * compares codes by the number of differing bits.
 *
 * The forward model of Section 2.1 (Eq. 1-2, reaction-diffusion with no-flux
 * boundary) is an explicit finite-difference scheme; its reading is stated
 * with its code at the end of this file.
 *
 * The nearest-neighbour downsampling of Section 2.3 (an order-0 spline
 * resampling to 64^3 or 32^3) is out[i] = in[f*i] along each axis.
 *
 * Volume layout everywhere: [nz][ny][nx], x fastest; voxel linear index
 * i = x + nx*(y + ny*z).
 *
 * Parity pins (tests/test_oracle_*.py): hand-worked 2x2x2 cases, Dice(A,A)=1,
 * disjoint masks give 0, symmetry, the Jaccard identity D = 2J/(1+J) computed
 * through Python sets, exact rationals for the score, planted duplicates for
 * the order, all 65,536 binary16 patterns against numpy's decoder, and
 * single-voxel volumes for the block-mean layout.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* IEEE 754 binary16 -> binary64, from the format's definition.         */
/* ------------------------------------------------------------------ */
double oracle_f16_to_f64(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int expo = (h >> 10) & 0x1F;
    int frac = h & 0x3FF;
    double mag;
    if (expo == 0) {
        mag = ldexp((double)frac, -24);               /* subnormal: frac * 2^-14 * 2^-10 */
    } else if (expo == 31) {
        mag = (frac == 0) ? INFINITY : NAN;
    } else {
        mag = ldexp((double)(1024 + frac), expo - 25); /* (1 + frac/1024) * 2^(expo-15) */
    }
    return sign ? -mag : mag;
}

/* Membership of one voxel in a thresholded segmentation (Section 2.3). */
static int in_mask_f32(float c, float t) { return c >= t; }
static int in_mask_f16(uint16_t h, float t)
{
    /* the binary16 value is exact in binary32, so comparing in binary64 is
       the same as comparing in binary32 */
    return oracle_f16_to_f64(h) >= (double)t;
}

/* Dice coefficient from exact counts; both masks empty -> 1. */
double oracle_dice(uint32_t inter, uint32_t size_a, uint32_t size_b)
{
    uint32_t denom = size_a + size_b;
    if (denom == 0) return 1.0;
    return (double)(2u * inter) / (double)denom;
}

/* Combined score: mean of Dice_T1Gd and Dice_FLAIR. */
double oracle_score(uint32_t i1, uint32_t i2, uint32_t e1, uint32_t e2,
                    uint32_t p1, uint32_t p2)
{
    double d1 = oracle_dice(i1, p1, e1);
    double d2 = oracle_dice(i2, p2, e2);
    return (d1 + d2) * 0.5;
}

/* ------------------------------------------------------------------ */
/* Patient segmentations as byte masks [2][v] (0/1).                    */
/* ------------------------------------------------------------------ */
void oracle_threshold_f32(const float* vol, int64_t v, float t1, float t2,
                          uint8_t* mask /* [2][v] */)
{
    for (int64_t x = 0; x < v; ++x) {
        mask[x] = (uint8_t)in_mask_f32(vol[x], t1);
        mask[v + x] = (uint8_t)in_mask_f32(vol[x], t2);
    }
}

void oracle_threshold_f16(const uint16_t* vol, int64_t v, float t1, float t2,
                          uint8_t* mask /* [2][v] */)
{
    for (int64_t x = 0; x < v; ++x) {
        mask[x] = (uint8_t)in_mask_f16(vol[x], t1);
        mask[v + x] = (uint8_t)in_mask_f16(vol[x], t2);
    }
}

/* Unpack the library's bit-plane format into byte masks: word w, bit b of a
   plane holds voxel 32*w + b.  planes is [2][words]. */
void oracle_unpack_planes(const uint32_t* planes, int64_t words, int64_t v,
                          uint8_t* mask /* [2][v] */)
{
    for (int k = 0; k < 2; ++k)
        for (int64_t x = 0; x < v; ++x)
            mask[k * v + x] = (uint8_t)((planes[k * words + x / 32] >> (x % 32)) & 1u);
}

/* ------------------------------------------------------------------ */
/* Per-entry counts: out[e] = {I1, I2, E1, E2}.                          */
/* The patient is given as its byte masks [2][v]; P_k is their sum.       */
/* ------------------------------------------------------------------ */
static void patient_sizes(const uint8_t* pmask, int64_t v, uint32_t* pcount)
{
    pcount[0] = pcount[1] = 0;
    for (int64_t x = 0; x < v; ++x) {
        pcount[0] += pmask[x];
        pcount[1] += pmask[v + x];
    }
}

int oracle_counts_f32(const float* db, int64_t n, int64_t v, const uint8_t* pmask,
                      float t1, float t2, int nthreads,
                      uint32_t* out /* [n][4] */, uint32_t* pcount /* [2] */)
{
    patient_sizes(pmask, v, pcount);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t e = 0; e < n; ++e) {
        const float* c = db + e * v;
        uint32_t i1 = 0, i2 = 0, e1 = 0, e2 = 0;
        for (int64_t x = 0; x < v; ++x) {
            int m1 = in_mask_f32(c[x], t1);
            int m2 = in_mask_f32(c[x], t2);
            e1 += m1;
            e2 += m2;
            i1 += m1 & pmask[x];
            i2 += m2 & pmask[v + x];
        }
        out[4 * e + 0] = i1;
        out[4 * e + 1] = i2;
        out[4 * e + 2] = e1;
        out[4 * e + 3] = e2;
    }
    (void)nthreads;
    return 0;
}

int oracle_counts_f16(const uint16_t* db, int64_t n, int64_t v, const uint8_t* pmask,
                      float t1, float t2, int nthreads,
                      uint32_t* out /* [n][4] */, uint32_t* pcount /* [2] */)
{
    patient_sizes(pmask, v, pcount);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t e = 0; e < n; ++e) {
        const uint16_t* c = db + e * v;
        uint32_t i1 = 0, i2 = 0, e1 = 0, e2 = 0;
        for (int64_t x = 0; x < v; ++x) {
            int m1 = in_mask_f16(c[x], t1);
            int m2 = in_mask_f16(c[x], t2);
            e1 += m1;
            e2 += m2;
            i1 += m1 & pmask[x];
            i2 += m2 & pmask[v + x];
        }
        out[4 * e + 0] = i1;
        out[4 * e + 1] = i2;
        out[4 * e + 2] = e1;
        out[4 * e + 3] = e2;
    }
    (void)nthreads;
    return 0;
}

/* Counts against database entries given directly as byte masks [n][2][v]
   (used for the downsampled loop and for masks built by other means).  A
   mask byte is a set membership, 0 or 1; any other byte value is rejected
   (returns -1, nothing written) because summing it would miscount. */
int oracle_counts_masks(const uint8_t* dbmask, int64_t n, int64_t v, const uint8_t* pmask,
                        int nthreads, uint32_t* out /* [n][4] */, uint32_t* pcount)
{
    for (int64_t x = 0; x < 2 * v; ++x)
        if (pmask[x] > 1) return -1;
    for (int64_t x = 0; x < n * 2 * v; ++x)
        if (dbmask[x] > 1) return -1;
    patient_sizes(pmask, v, pcount);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t e = 0; e < n; ++e) {
        const uint8_t* m = dbmask + e * 2 * v;
        uint32_t i1 = 0, i2 = 0, e1 = 0, e2 = 0;
        for (int64_t x = 0; x < v; ++x) {
            e1 += m[x];
            e2 += m[v + x];
            i1 += m[x] & pmask[x];
            i2 += m[v + x] & pmask[v + x];
        }
        out[4 * e + 0] = i1;
        out[4 * e + 1] = i2;
        out[4 * e + 2] = e1;
        out[4 * e + 3] = e2;
    }
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ranking: (score descending, index ascending), first k.               */
/* ------------------------------------------------------------------ */
typedef struct { double score; int64_t index; } ranked;

static int ranked_cmp(const void* pa, const void* pb)
{
    const ranked* a = (const ranked*)pa;
    const ranked* b = (const ranked*)pb;
    if (a->score > b->score) return -1;
    if (a->score < b->score) return 1;
    if (a->index < b->index) return -1;
    if (a->index > b->index) return 1;
    return 0;
}

/* scores[n] -> out_index[k], out_score[k].  Returns 0, or -1 if k > n. */
int oracle_rank(const double* scores, int64_t n, int64_t k,
                int64_t* out_index, double* out_score)
{
    if (k > n || k < 0) return -1;
    ranked* r = (ranked*)malloc(sizeof(ranked) * (size_t)(n > 0 ? n : 1));
    if (!r) return -2;
    for (int64_t e = 0; e < n; ++e) { r[e].score = scores[e]; r[e].index = e; }
    qsort(r, (size_t)n, sizeof(ranked), ranked_cmp);
    for (int64_t j = 0; j < k; ++j) { out_index[j] = r[j].index; out_score[j] = r[j].score; }
    free(r);
    return 0;
}

/* Scores for all entries from their counts. */
void oracle_scores(const uint32_t* counts /* [n][4] */, int64_t n, const uint32_t* pcount,
                   double* scores /* [n] */)
{
    for (int64_t e = 0; e < n; ++e)
        scores[e] = oracle_score(counts[4 * e + 0], counts[4 * e + 1],
                                 counts[4 * e + 2], counts[4 * e + 3],
                                 pcount[0], pcount[1]);
}

/* ------------------------------------------------------------------ */
/* Low-dimensional representations.                                     */
/* ------------------------------------------------------------------ */

/* Block mean of a byte mask over f x f x f blocks (nx, ny, nz multiples of f):
   out[bx + (nx/f)*(by + (ny/f)*bz)] = (1/f^3) * #{voxels set in the block}. */
int oracle_block_mean(const uint8_t* mask, int nx, int ny, int nz, int f, double* out)
{
    if (f <= 0 || nx % f || ny % f || nz % f) return -1;
    int bx_n = nx / f, by_n = ny / f, bz_n = nz / f;
    for (int bz = 0; bz < bz_n; ++bz)
        for (int by = 0; by < by_n; ++by)
            for (int bx = 0; bx < bx_n; ++bx) {
                int64_t count = 0;
                for (int z = bz * f; z < (bz + 1) * f; ++z)
                    for (int y = by * f; y < (by + 1) * f; ++y)
                        for (int x = bx * f; x < (bx + 1) * f; ++x)
                            count += mask[(int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z)];
                out[bx + bx_n * (by + by_n * bz)] = (double)count / ((double)f * f * f);
            }
    return 0;
}

/* bfloat16 encoding of a binary32 value: round to nearest-even at bit 16.
   Returns the bit pattern; NaN/Inf are not produced by the callers. */
uint16_t oracle_bf16_bits(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    uint32_t lsb = (b >> 16) & 1u;
    b += 0x7FFFu + lsb;
    return (uint16_t)(b >> 16);
}

double oracle_bf16_value(uint16_t h)
{
    uint32_t b = (uint32_t)h << 16;
    float f;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* FP8 E4M3 value of code c (sign, 4-bit exponent with bias 7, 3-bit fraction;
   exponent 15 with fraction 7 is NaN). */
double oracle_e4m3_value(uint8_t c)
{
    int sign = (c >> 7) & 1;
    int expo = (c >> 3) & 0xF;
    int frac = c & 0x7;
    double mag;
    if (expo == 15 && frac == 7) return NAN;
    if (expo == 0) mag = ldexp((double)frac, -9);             /* frac/8 * 2^-6 */
    else mag = ldexp((double)(8 + frac), expo - 10);          /* (1+frac/8) * 2^(expo-7) */
    return sign ? -mag : mag;
}

/* FP8 E4M3 code nearest to x (ties to even code), saturating at +-448:
   searched over all finite codes of x's sign -- slow and plain. */
uint8_t oracle_e4m3_code(double x)
{
    int neg = signbit(x) ? 1 : 0;
    double a = fabs(x);
    if (a >= 448.0) return (uint8_t)((neg << 7) | 0x7E);
    uint8_t best = 0;
    double best_err = INFINITY;
    for (int c = 0; c < 0x7F; ++c) {                /* 0x7F is NaN */
        double v = oracle_e4m3_value((uint8_t)c);
        double err = fabs(v - a);
        if (err < best_err || (err == best_err && (c & 1) == 0)) {
            best_err = err;
            best = (uint8_t)c;
        }
    }
    return (uint8_t)((neg << 7) | best);
}

/* Embedding of one byte mask: f^3 block counts / f^3 (exact in binary32),
   encoded as bfloat16 and as FP8 E4M3 with the row scale s (see header).
   out_bf16[d], out_e4m3[d], out_scale[1]; returns d or -1. */
int oracle_embed(const uint8_t* mask, int nx, int ny, int nz, int f,
                 uint16_t* out_bf16, uint8_t* out_e4m3, float* out_scale)
{
    if (f <= 0 || nx % f || ny % f || nz % f) return -1;
    int d = (nx / f) * (ny / f) * (nz / f);
    double* mean = (double*)malloc(sizeof(double) * (size_t)d);
    if (!mean) return -1;
    oracle_block_mean(mask, nx, ny, nz, f, mean);
    float m = 0.0f;
    for (int j = 0; j < d; ++j) {
        float e = (float)mean[j];                   /* count / f^3, exact */
        out_bf16[j] = oracle_bf16_bits(e);
        if (e > m) m = e;
    }
    float s = (m == 0.0f) ? 1.0f : m / 448.0f;
    for (int j = 0; j < d; ++j) {
        float e = (float)mean[j];
        float r = e / s;                            /* binary32, as the kernel divides */
        out_e4m3[j] = oracle_e4m3_code((double)r);
    }
    *out_scale = s;
    free(mean);
    return d;
}

/* SplitMix64 output for counter value i of a stream with key k: the
   finaliser applied to k + (i + 1) * 0x9E3779B97F4A7C15. */
uint64_t oracle_splitmix64(uint64_t key, uint64_t i)
{
    uint64_t z = key + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Count sketch of one byte mask [v] into d buckets (d a power of two):
   out[h mod d] += (bit 31 of h ? -1 : +1) for every set voxel x, with
   h = oracle_splitmix64(0, x) >> 32 for the bucket and the whole h for the
   sign.  Returns 0, or -1 if d is not a power of two. */
int oracle_sketch(const uint8_t* mask, int64_t v, int d, int32_t* out)
{
    if (d <= 0 || (d & (d - 1))) return -1;
    for (int j = 0; j < d; ++j) out[j] = 0;
    for (int64_t x = 0; x < v; ++x) {
        if (!mask[x]) continue;
        const uint64_t h = oracle_splitmix64(0, (uint64_t)x);
        const int bucket = (int)((h >> 32) & (uint64_t)(d - 1));
        out[bucket] += ((h >> 31) & 1u) ? -1 : 1;
    }
    return 0;
}

/* Sign code of a sketch: bit j of word j/32 is [v_j > 0]. */
void oracle_sign_code(const int32_t* sk, int d, uint32_t* code /* [d/32] */)
{
    for (int w = 0; w < d / 32; ++w) code[w] = 0;
    for (int j = 0; j < d; ++j)
        if (sk[j] > 0) code[j / 32] |= 1u << (j % 32);
}

/* Number of differing bits of two codes of `words` words. */
int64_t oracle_hamming(const uint32_t* a, const uint32_t* b, int64_t words)
{
    int64_t h = 0;
    for (int64_t w = 0; w < words; ++w) {
        uint32_t x = a[w] ^ b[w];
        while (x) {
            h += x & 1u;
            x >>= 1;
        }
    }
    return h;
}

/* Euclidean distance between two vectors of length d, in binary64. */
double oracle_l2(const double* a, const double* b, int64_t d)
{
    double s = 0.0;
    for (int64_t j = 0; j < d; ++j) {
        double diff = a[j] - b[j];
        s += diff * diff;
    }
    return sqrt(s);
}

/* Nearest-neighbour (order-0 spline) downsampling by integer factor f:
   out[x + (nx/f)*(y + (ny/f)*z)] = in[f*x + nx*(f*y + ny*f*z)]. */
int oracle_downsample_nn_u8(const uint8_t* in, int nx, int ny, int nz, int f, uint8_t* out)
{
    if (f <= 0 || nx % f || ny % f || nz % f) return -1;
    int ox = nx / f, oy = ny / f, oz = nz / f;
    for (int z = 0; z < oz; ++z)
        for (int y = 0; y < oy; ++y)
            for (int x = 0; x < ox; ++x)
                out[x + (int64_t)ox * (y + (int64_t)oy * z)] =
                    in[(int64_t)f * x + (int64_t)nx * ((int64_t)f * y + (int64_t)ny * ((int64_t)f * z))];
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Forward model of Section 2.1 (Eq. 1-2): the reaction-diffusion equation
 *   du/dt = div(D grad u) + rho u (1 - u)   in the brain Omega,
 *   n . grad u = 0                           on its boundary,
 *   u(r, 0) = u0 at the seed voxel r*, 0 elsewhere.
 *
 * The paper names no discretisation; the reading taken here:
 *   * a voxel grid of unit spacing; D(x) = D_w m(x) with m the tissue's
 *     relative diffusivity (the caller's map; Omega = {m > 0});
 *   * the flux through the face between neighbours i and j is
 *     D_w h(m_i, m_j) (u_j - u_i), h the harmonic mean 2 m_i m_j / (m_i + m_j);
 *     h = 0 when either voxel is outside Omega, which is the no-flux
 *     condition of Eq. 2 on the domain's boundary; faces on the edge of the
 *     grid carry no flux either;
 *   * explicit Euler in time, every voxel from the previous step's values:
 *     u_i <- u_i + dt (D_w sum_j h(m_i, m_j) (u_j - u_i) + rho u_i (1 - u_i)),
 *     the six neighbours taken in the order -x, +x, -y, +y, -z, +z;
 *   * n = ceil(T_end (6 D_w max(m) + rho) / cfl) steps of dt = T_end / n
 *     (n = 0 for T_end = 0; 0 < cfl <= 1 keeps 0 <= u <= 1);
 *   * the seed voxel is the nearest voxel to (x, y, z): floor(c + 0.5).
 * Everything is binary64.
 * ------------------------------------------------------------------------ */
static double rd_face(double a, double b)
{
    return (a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
}

int64_t oracle_rd_steps(double t_end, double dw, double rho, double m_max, double cfl)
{
    if (!(t_end > 0.0)) return 0;
    double rate = 6.0 * dw * m_max + rho;
    double n = ceil(t_end * rate / cfl);
    return n < 1.0 ? 1 : (int64_t)n;
}

/* theta = (x, y, z, D_w, rho, T_end).  out [nz][ny][nx] binary64 = u(T_end).
   Returns the number of steps, or -1 for a seed outside the grid or the
   domain, or an invalid parameter. */
int64_t oracle_rd_simulate(const float* tissue, int nx, int ny, int nz, const double* theta,
                           double u0, double cfl, double* out)
{
    const int64_t v = (int64_t)nx * ny * nz;
    const double dw = theta[3], rho = theta[4], t_end = theta[5];
    if (!(cfl > 0.0 && cfl <= 1.0) || !(dw >= 0.0) || !(rho >= 0.0) || !(t_end >= 0.0))
        return -1;
    const double fx = floor(theta[0] + 0.5), fy = floor(theta[1] + 0.5), fz = floor(theta[2] + 0.5);
    if (fx < 0 || fy < 0 || fz < 0 || fx >= nx || fy >= ny || fz >= nz) return -1;
    const int64_t seed = (int64_t)fx + (int64_t)nx * ((int64_t)fy + (int64_t)ny * (int64_t)fz);
    if (!(tissue[seed] > 0.0f)) return -1;
    double m_max = 0.0;
    for (int64_t i = 0; i < v; ++i)
        if ((double)tissue[i] > m_max) m_max = (double)tissue[i];
    const int64_t n = oracle_rd_steps(t_end, dw, rho, m_max, cfl);
    const double dt = n ? t_end / (double)n : 0.0;
    double* u = (double*)calloc((size_t)v, sizeof(double));
    double* w = (double*)calloc((size_t)v, sizeof(double));
    if (!u || !w) {
        free(u);
        free(w);
        return -1;
    }
    u[seed] = u0;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    for (int64_t step = 0; step < n; ++step) {
        /* voxels of one step are independent: spread the planes over cores */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const int64_t i = x + sy * y + sz * z;
                    const double ui = u[i], mi = tissue[i];
                    double flux = 0.0;
                    if (x > 0) flux += rd_face(mi, tissue[i - 1]) * (u[i - 1] - ui);
                    if (x < nx - 1) flux += rd_face(mi, tissue[i + 1]) * (u[i + 1] - ui);
                    if (y > 0) flux += rd_face(mi, tissue[i - sy]) * (u[i - sy] - ui);
                    if (y < ny - 1) flux += rd_face(mi, tissue[i + sy]) * (u[i + sy] - ui);
                    if (z > 0) flux += rd_face(mi, tissue[i - sz]) * (u[i - sz] - ui);
                    if (z < nz - 1) flux += rd_face(mi, tissue[i + sz]) * (u[i + sz] - ui);
                    w[i] = ui + dt * (dw * flux + rho * ui * (1.0 - ui));
                }
        double* t = u;
        u = w;
        w = t;
    }
    memcpy(out, u, (size_t)v * sizeof(double));
    free(u);
    free(w);
    return n;
}
