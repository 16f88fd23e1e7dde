/*
 * CPU oracle for brushed multivariate volume rendering and linked
 * parallel-coordinates histograms (arXiv 2207.12011, Section 2.2 "Rendering"
 * and Section 2.1 "Data Preprocessing").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this file;
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it. It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes, plainly and slowly:
 *   - brick min/max per variable over each 8^3 brick plus its +1 apron;
 *   - brush classification of bricks (shell intersection and brush box)
 *     and of interpolation cells (every sample fails / passes / must be
 *     interpolated);
 *   - the 2x2x2 mean used for the coarser levels of detail (Section 2.1);
 *   - progressive passes with a per-pixel jittered lattice offset;
 *   - front-to-back emission-absorption ray marching where a sample is
 *     discarded when any restricted variable lies outside its brush bounds
 *     (Section 2.2), colour from a 1D transfer function, early termination;
 *   - adjacent-axis parallel-coordinates density histograms of the in-shell,
 *     in-brush cells (Section 2.1 PC data, Fig. 2);
 *   - implicit position axes (x, y, z and radius of a sample or cell centre)
 *     as brush and PC axes (Section 2.1 derived altitude, Section 3 cuts on
 *     Cartesian coordinates);
 *   - the random subsample of cells whose polylines the PC plot draws
 *     (Section 2.1);
 *   - the brush test of given points (pathline seeds inside the current
 *     selection, Section 3);
 *   - image warping of a rendered frame to a new camera (Section 2.2).
 *
 * Precision. Every continuous quantity (ray geometry for the colour value,
 * transfer-function lookup, opacity, compositing) is FP64. Every quantity that
 * DECIDES an integer -- how many lattice samples a ray has, whether a sample
 * is in the shell, which cell it interpolates from, whether its FP32
 * trilinear value passes the brush, which bricks are active -- is computed in
 * FP32 with individually rounded IEEE operations (fmaf, +, -, *, /, sqrtf) in
 * one fixed order, because the method interpolates in software FP32 and an
 * integer decision must be taken in the precision of the method on both sides.
 * Build with -ffp-contract=off so the compiler fuses nothing on its own.
 *
 * Parity of the appearance against the paper's figures is unpinned: the
 * figures and the data set are absent.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------ */
/* Volume access: vol[v][z][y][x] float32 (stored values, exact).       */
/* ------------------------------------------------------------------ */
static inline float val(const float *vol, int n, int v, int x, int y, int z) {
    return vol[(((size_t)v * n + z) * n + y) * n + x];
}

/* ------------------------------------------------------------------ */
/* Brick min/max: for brick (bx,by,bz) of edge bs cells and variable v,  */
/* the min and max of the stored values at vertices bs*b .. min(bs*b+bs, */
/* n-1) on each axis. A sample whose lower interpolation corner lies in  */
/* the brick reads only these vertices. NaN values are ignored.          */
/* Output layout: [bz][by][bx][v].                                      */
/* ------------------------------------------------------------------ */
void oracle_brick_minmax(const float *vol, int n, int nvars, int bs, float *out_min, float *out_max) {
    const int BRICK = bs;
    int nb = (n + BRICK - 1) / BRICK;
    for (int bz = 0; bz < nb; bz++)
        for (int by = 0; by < nb; by++)
            for (int bx = 0; bx < nb; bx++)
                for (int v = 0; v < nvars; v++) {
                    double mn = NAN, mx = NAN;
                    int x1 = bx * BRICK + BRICK; if (x1 > n - 1) x1 = n - 1;
                    int y1 = by * BRICK + BRICK; if (y1 > n - 1) y1 = n - 1;
                    int z1 = bz * BRICK + BRICK; if (z1 > n - 1) z1 = n - 1;
                    for (int z = bz * BRICK; z <= z1; z++)
                        for (int y = by * BRICK; y <= y1; y++)
                            for (int x = bx * BRICK; x <= x1; x++) {
                                double a = val(vol, n, v, x, y, z);
                                mn = fmin(mn, a);
                                mx = fmax(mx, a);
                            }
                    size_t o = (((size_t)bz * nb + by) * nb + bx) * nvars + v;
                    out_min[o] = (float)mn;
                    out_max[o] = (float)mx;
                }
}

/* ------------------------------------------------------------------ */
/* Brush classification of bricks of edge bs (FP32 decisions).          */
/*                                                                      */
/* A brick is active when (1) the world box its samples can occupy,     */
/* widened by 2^-10, meets the shell r_in <= |p| <= r_out, and (2) for   */
/* every restricted variable v, max_v + d >= lo_v and min_v - d <= hi_v, */
/* d = max(|min_v|, |max_v|) * 2^-20 + 2^-120. The widening d covers     */
/* the rounding of the FP32 trilinear interpolation (at most about      */
/* 10 * 2^-24 * max|corner|), so no sample that passes the brush can    */
/* lie in an inactive brick. A variable with max(|min_v|, |max_v|) >    */
/* 2^126 never deactivates a brick: a corner difference can overflow    */
/* there and the interpolated value can be infinite. A brick is         */
/* skippable when it and all its existing 26 neighbours are inactive.   */
/* Implicit position axes (Section 2.1 derives altitude, Section 3 cuts   */
/* the volume on Cartesian coordinates). Axis a of a point p: a = 0, 1, 2 */
/* the coordinate p[a]; a = 3 the radius sqrtf(fmaf(z, z, fmaf(y, y,     */
/* x * x))). A position brush restricts axis a (bit a of pmask) to       */
/* plo[a] <= value <= phi[a]. In PC axis lists, axis id 8 + a names      */
/* position axis a (ids 0..nvars-1 name stored variables).               */
/* The position of a sample is its FP32 lattice point; that of a cell is */
/* its centre, coordinate (float)(2i + 1 - n) / (float)n.                */
/* ------------------------------------------------------------------ */
static float sq3_f32(const float p[3]) {
    return fmaf(p[2], p[2], fmaf(p[1], p[1], p[0] * p[0]));
}

static float pos_axis(const float p[3], int a) {
    return a < 3 ? p[a] : sqrtf(sq3_f32(p));
}

static int pos_pass(const float p[3], const float *plo, const float *phi, uint32_t pmask) {
    for (int a = 0; a < 4; a++) {
        if (!((pmask >> a) & 1u)) continue;
        float v = pos_axis(p, a);
        if (!(v >= plo[a] && v <= phi[a])) return 0;
    }
    return 1;
}

static void cell_centre(int n, int x, int y, int z, float p[3]) {
    p[0] = (float)(2 * x + 1 - n) / (float)n;
    p[1] = (float)(2 * y + 1 - n) / (float)n;
    p[2] = (float)(2 * z + 1 - n) / (float)n;
}

/* ------------------------------------------------------------------ */
/* Brick classification. A brick is active iff its widened sample box   */
/* meets the shell, every restricted variable's range can pass, and the */
/* box can meet the position brush: for a = 0..2 the box's [l_a, h_a]   */
/* meets [plo_a, phi_a]; for the radius sqrtf(far^2) >= plo_3 and        */
/* sqrtf(near^2) <= phi_3 (near/far: the box's closest and farthest     */
/* corner distances, squared with the same FP32 chain as a sample's).   */
/* The squared-distance chain is monotone in each |coordinate| and       */
/* sqrtf is monotone, so no sample of an inactive brick passes.          */
/* Output: active[b], skippable[b] as bytes 0/1, b = (bz*nb+by)*nb+bx.  */
/* ------------------------------------------------------------------ */
static void brick_box_axis(int b, int nb, int n, int BRICK, float *lo, float *hi) {
    float sc = 2.0f / (float)n;
    float l = fmaf((float)(b * BRICK) + 0.5f, sc, -1.0f) - 0x1p-10f;
    float h = fmaf((float)(b * BRICK + BRICK) + 0.5f, sc, -1.0f) + 0x1p-10f;
    if (b == 0) l = -2.0f;
    if (b == nb - 1) h = 2.0f;
    *lo = l;
    *hi = h;
}

void oracle_classify(const float *bmin, const float *bmax, int n, int nvars, int bs,
                     float r_in, float r_out, const float *lo, const float *hi,
                     uint32_t active_mask, const float *plo, const float *phi, uint32_t pmask,
                     uint8_t *active, uint8_t *skippable) {
    const int BRICK = bs;
    int nb = (n + BRICK - 1) / BRICK;
    float rin2 = r_in * r_in, rout2 = r_out * r_out;
    for (int bz = 0; bz < nb; bz++)
        for (int by = 0; by < nb; by++)
            for (int bx = 0; bx < nb; bx++) {
                int bc[3] = {bx, by, bz};
                float nearc[3], farc[3];
                int act = 1;
                for (int a = 0; a < 3; a++) {
                    float l, h;
                    brick_box_axis(bc[a], nb, n, BRICK, &l, &h);
                    nearc[a] = (l > 0.0f) ? l : ((h < 0.0f) ? -h : 0.0f);
                    farc[a] = fmaxf(fabsf(l), fabsf(h));
                    if (((pmask >> a) & 1u) && !(h >= plo[a] && l <= phi[a])) act = 0;
                }
                float near2 = sq3_f32(nearc);
                float far2 = sq3_f32(farc);
                act = act && (near2 <= rout2) && (far2 >= rin2);
                if (((pmask >> 3) & 1u) && !(sqrtf(far2) >= plo[3] && sqrtf(near2) <= phi[3])) act = 0;
                size_t b = ((size_t)bz * nb + by) * nb + bx;
                for (int v = 0; v < nvars && act; v++) {
                    if (!((active_mask >> v) & 1u)) continue;
                    float mn = bmin[b * nvars + v], mx = bmax[b * nvars + v];
                    float m = fmaxf(fabsf(mn), fabsf(mx));
                    if (m > 0x1p126f) continue;
                    float d = fmaf(m, 0x1p-20f, 0x1p-120f);
                    float up = mx + d, dn = mn - d;
                    if (!(up >= lo[v] && dn <= hi[v])) act = 0;
                }
                active[b] = (uint8_t)act;
            }
    for (int bz = 0; bz < nb; bz++)
        for (int by = 0; by < nb; by++)
            for (int bx = 0; bx < nb; bx++) {
                int s = 1;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            int x = bx + dx, y = by + dy, z = bz + dz;
                            if (x < 0 || y < 0 || z < 0 || x >= nb || y >= nb || z >= nb) continue;
                            if (active[((size_t)z * nb + y) * nb + x]) s = 0;
                        }
                skippable[((size_t)bz * nb + by) * nb + bx] = (uint8_t)s;
            }
}

/* ------------------------------------------------------------------ */
/* Cell classes under a brush (FP32 decisions). For the interpolation   */
/* cell with lower corner (x,y,z), 0 <= x,y,z <= n-2, and each          */
/* restricted variable v, over its 8 corner values:                     */
/*   FAIL   if a corner is NaN (the trilinear value is NaN), or, with    */
/*          m = max(|min|,|max|) <= 2^126 and d as for bricks,          */
/*          max + d < lo_v or min - d > hi_v (every value fails v);     */
/*   INSIDE if m <= 2^126, min - d >= lo_v and max + d <= hi_v (every   */
/*          value passes v);                                            */
/*   MIXED  otherwise (the value must be interpolated).                 */
/* The 2^126 bound keeps the FP32 interpolation free of overflow, and d */
/* covers its rounding (at most about 9 * 2^-24 * m), so FAIL and       */
/* INSIDE are exact statements about the FP32 trilinear value of every  */
/* sample whose lower interpolation corner is (x,y,z).                  */
/* Output word per cell: bit v set iff v is MIXED, bit 15 set iff some  */
/* restricted v is FAIL; [z][y][x] over n^3 cells, 0 where an index is  */
/* n-1 (no such cell).                                                   */
/* ------------------------------------------------------------------ */
void oracle_cell_classes(const float *vol, int n, int nvars, const float *lo, const float *hi,
                         uint32_t active_mask, uint16_t *out) {
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                uint16_t word = 0;
                if (x < n - 1 && y < n - 1 && z < n - 1) {
                    for (int v = 0; v < nvars; v++) {
                        if (!((active_mask >> v) & 1u)) continue;
                        int has_nan = 0;
                        float mn = INFINITY, mx = -INFINITY;
                        for (int c = 0; c < 8; c++) {
                            float a = val(vol, n, v, x + (c & 1), y + ((c >> 1) & 1), z + (c >> 2));
                            if (a != a) has_nan = 1;
                            else {
                                if (a < mn) mn = a;
                                if (a > mx) mx = a;
                            }
                        }
                        if (has_nan) { word |= 0x8000u; continue; }
                        float m = fmaxf(fabsf(mn), fabsf(mx));
                        if (m > 0x1p126f) { word |= (uint16_t)(1u << v); continue; }
                        float d = fmaf(m, 0x1p-20f, 0x1p-120f);
                        float up = mx + d, dn = mn - d;
                        if (up < lo[v] || dn > hi[v]) word |= 0x8000u;
                        else if (!(dn >= lo[v] && up <= hi[v])) word |= (uint16_t)(1u << v);
                    }
                }
                out[((size_t)z * n + y) * n + x] = word;
            }
}

/* ------------------------------------------------------------------ */
/* Level of detail (Section 2.1: each coarser level holds 1/8 of the    */
/* cells). Coarse cell (i,j,k) = mean of fine cells (2i+a, 2j+b, 2k+c), */
/* a,b,c in {0,1}, fine indices clamped to n-1; summed in FP32 as       */
/* ((c000+c100)+(c010+c110)) + ((c001+c101)+(c011+c111)), times 1/8.    */
/* Output: [v][m][m][m] float32, m = (n+1)/2.                           */
/* ------------------------------------------------------------------ */
void oracle_lod_mean(const float *vol, int n, int nvars, float *out) {
    int m = (n + 1) / 2;
    for (int v = 0; v < nvars; v++)
        for (int k = 0; k < m; k++)
            for (int j = 0; j < m; j++)
                for (int i = 0; i < m; i++) {
                    int x0 = 2 * i, y0 = 2 * j, z0 = 2 * k;
                    int x1 = x0 + 1 < n ? x0 + 1 : n - 1;
                    int y1 = y0 + 1 < n ? y0 + 1 : n - 1;
                    int z1 = z0 + 1 < n ? z0 + 1 : n - 1;
                    float s0 = (val(vol, n, v, x0, y0, z0) + val(vol, n, v, x1, y0, z0)) +
                               (val(vol, n, v, x0, y1, z0) + val(vol, n, v, x1, y1, z0));
                    float s1 = (val(vol, n, v, x0, y0, z1) + val(vol, n, v, x1, y0, z1)) +
                               (val(vol, n, v, x0, y1, z1) + val(vol, n, v, x1, y1, z1));
                    out[(((size_t)v * m + k) * m + j) * m + i] = (s0 + s1) * 0.125f;
                }
}

/* ------------------------------------------------------------------ */
/* Parallel-coordinates histograms.                                     */
/*                                                                      */
/* Cell (x,y,z) of an n^3 grid has centre p = (2i+1-n)/n per axis. It  */
/* is in the shell iff S_in <= s <= S_out with the integer              */
/* s = sum (2i+1-n)^2, S_in = ceil((r_in n)^2), S_out = floor((r_out n)^2)*/
/* (both evaluated in double). It is in the brush iff lo_v <= v <= hi_v */
/* for every restricted v (NaN fails). Its bin on an axis is the number */
/* of interior edges e_1..e_{bins-1} that are <= the value. For each     */
/* adjacent axis pair p: H[p][bin_p][bin_{p+1}] += 1.                    */
/* ------------------------------------------------------------------ */
void oracle_shell_bounds(int n, float r_in, float r_out, int64_t *s_in, int64_t *s_out) {
    double a = (double)r_in * (double)n, b = (double)r_out * (double)n;
    *s_in = (int64_t)ceil(a * a);
    *s_out = (int64_t)floor(b * b);
}

static int bin_of(float v, const float *edges, int bins) {
    int c = 0;
    for (int k = 1; k < bins; k++)
        if (v >= edges[k]) c++;
    return c;
}

/* Value of PC axis id `axis` at cell (x, y, z): a stored variable, or  */
/* (id 8 + a) position axis a at the cell centre.                         */
static float cell_axis(const float *vol, int n, int axis, int x, int y, int z) {
    if (axis < 8) return val(vol, n, axis, x, y, z);
    float p[3];
    cell_centre(n, x, y, z, p);
    return pos_axis(p, axis - 8);
}

/* In-brush test of a cell: restricted stored values and the position    */
/* brush at the cell centre.                                              */
static int cell_in_brush(const float *vol, int n, int nvars, const float *lo, const float *hi,
                         uint32_t active_mask, const float *plo, const float *phi, uint32_t pmask,
                         int x, int y, int z) {
    for (int v = 0; v < nvars; v++) {
        if (!((active_mask >> v) & 1u)) continue;
        float a = val(vol, n, v, x, y, z);
        if (!(a >= lo[v] && a <= hi[v])) return 0;
    }
    if (pmask) {
        float p[3];
        cell_centre(n, x, y, z, p);
        if (!pos_pass(p, plo, phi, pmask)) return 0;
    }
    return 1;
}

void oracle_histogram(const float *vol, int n, int nvars, float r_in, float r_out,
                      const float *lo, const float *hi, uint32_t active_mask,
                      const float *plo, const float *phi, uint32_t pmask, int use_brush,
                      const int *axis_order, int naxes, int bins, const float *edges,
                      uint32_t *out /* (naxes-1)*bins*bins */, uint64_t *out_cells) {
    int64_t s_in, s_out;
    oracle_shell_bounds(n, r_in, r_out, &s_in, &s_out);
    memset(out, 0, sizeof(uint32_t) * (size_t)(naxes - 1) * bins * bins);
    uint64_t cells = 0;
    int *b = (int *)malloc(sizeof(int) * naxes);
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                int64_t dx = 2 * x + 1 - n, dy = 2 * y + 1 - n, dz = 2 * z + 1 - n;
                int64_t s = dx * dx + dy * dy + dz * dz;
                if (s < s_in || s > s_out) continue;
                if (use_brush && !cell_in_brush(vol, n, nvars, lo, hi, active_mask, plo, phi, pmask, x, y, z))
                    continue;
                cells++;
                for (int a = 0; a < naxes; a++)
                    b[a] = bin_of(cell_axis(vol, n, axis_order[a], x, y, z), edges + (size_t)a * (bins + 1), bins);
                for (int p = 0; p + 1 < naxes; p++)
                    out[((size_t)p * bins + b[p]) * bins + b[p + 1]] += 1u;
            }
    free(b);
    if (out_cells) *out_cells = cells;
}

/* ------------------------------------------------------------------ */
/* PC line data (Section 2.1: the plot draws the polylines of a random  */
/* subsample of at most 100 000 cells). Among the in-shell cells (the    */
/* histograms' integer test), take the min(k, N) cells with the          */
/* smallest keys K(c) = SplitMix64 output at the state                   */
/* (seed * 2^32 + 2^32 - 1) + (c + 1) * 0x9E3779B97F4A7C15, c =          */
/* (z*n + y)*n + x (the progressive passes use the states of pass        */
/* indices below 2^32 - 1). The output function is a bijection and the   */
/* increment is odd, so keys are distinct and the subsample is exactly    */
/* defined. Output in increasing c: the cell index, the values of the    */
/* given PC axes (stored variables or position axes), and whether the    */
/* cell passes the brush (stored values, position brush at the centre).  */
/* Returns the number of cells written, or -1 on bad arguments.          */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t cell; } keyed_cell;

static int by_key(const void *a, const void *b) {
    uint64_t x = ((const keyed_cell *)a)->key, y = ((const keyed_cell *)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int by_cell(const void *a, const void *b) {
    int64_t x = ((const keyed_cell *)a)->cell, y = ((const keyed_cell *)b)->cell;
    return x < y ? -1 : (x > y ? 1 : 0);
}

uint64_t oracle_splitmix64_output(uint64_t z);

uint64_t oracle_subsample_key(uint32_t seed, int64_t cell) {
    uint64_t key = ((uint64_t)seed << 32) | 0xFFFFFFFFull;
    return oracle_splitmix64_output(key + (uint64_t)(cell + 1) * 0x9E3779B97F4A7C15ULL);
}

int64_t oracle_pc_subsample(const float *vol, int n, int nvars, float r_in, float r_out,
                            const float *lo, const float *hi, uint32_t active_mask,
                            const float *plo, const float *phi, uint32_t pmask,
                            uint32_t seed, int64_t k, const int *axis_order, int naxes,
                            int64_t *out_cells, float *out_values, uint8_t *out_in_brush) {
    if (n < 1 || k < 0 || naxes < 0) return -1;
    int64_t s_in, s_out;
    oracle_shell_bounds(n, r_in, r_out, &s_in, &s_out);
    int64_t ncell = (int64_t)n * n * n, cnt = 0;
    keyed_cell *all = (keyed_cell *)malloc(sizeof(keyed_cell) * (size_t)(ncell > 0 ? ncell : 1));
    if (!all) return -1;
    for (int z = 0; z < n; z++)
        for (int y = 0; y < n; y++)
            for (int x = 0; x < n; x++) {
                int64_t dx = 2 * x + 1 - n, dy = 2 * y + 1 - n, dz = 2 * z + 1 - n;
                int64_t s = dx * dx + dy * dy + dz * dz;
                if (s < s_in || s > s_out) continue;
                int64_t c = ((int64_t)z * n + y) * n + x;
                all[cnt].key = oracle_subsample_key(seed, c);
                all[cnt].cell = c;
                cnt++;
            }
    qsort(all, (size_t)cnt, sizeof(keyed_cell), by_key);
    int64_t m = k < cnt ? k : cnt;
    qsort(all, (size_t)m, sizeof(keyed_cell), by_cell);
    for (int64_t i = 0; i < m; i++) {
        int64_t c = all[i].cell;
        int x = (int)(c % n), y = (int)((c / n) % n), z = (int)(c / ((int64_t)n * n));
        out_cells[i] = c;
        for (int a = 0; a < naxes; a++) out_values[i * naxes + a] = cell_axis(vol, n, axis_order[a], x, y, z);
        out_in_brush[i] = (uint8_t)cell_in_brush(vol, n, nvars, lo, hi, active_mask, plo, phi, pmask, x, y, z);
    }
    free(all);
    return m;
}

/* ------------------------------------------------------------------ */
/* Ray marching (Section 2.2).                                          */
/* ------------------------------------------------------------------ */
typedef struct {
    const float *vol;
    int n, nvars;
    float r_in, r_out;
    const float *cam;       /* eye[3], target[3], up[3], tan_half_vfov */
    int w, h;
    float dt;
    const float *lo, *hi;
    uint32_t active_mask;
    const float *plo, *phi; /* position brush (axes x, y, z, radius) */
    uint32_t pmask;
    const uint8_t *tfvis;   /* TF visibility of the 4^3 sub-bricks (NULL: no TF skipping) */
    int nsb;
    const float *tf;        /* 256 x (r,g,b,sigma) */
    int color_var;
    float tf_lo, tf_hi;
    const double *bg;       /* premultiplied background rgba */
    int ert;
    const int64_t *pixels;  /* NULL: all pixels in row-major order */
    int64_t npix;
    double *out;            /* npix x 4 */
    uint32_t *counts;       /* npix x 2: marched lattice samples, kept samples (may be NULL) */
    float *depth;           /* npix: FP32 t of the first kept sample, +inf if none (may be NULL) */
    uint32_t seed, pass;    /* progressive pass: lattice offset of every pixel (pass 0: 1/2) */
    int exact;              /* 1: every decision in FP64 on the plain definition (render_pixel_exact) */
    int64_t next;           /* shared work counter */
    pthread_mutex_t lock;
} render_job;

/* ------------------------------------------------------------------ */
/* Progressive passes (Section 2: passes keep refining the image while  */
/* the camera rests). Pass p >= 1 of a pixel places its lattice at      */
/* t_k = t0 + (k + j) dt instead of t0 + (k + 1/2) dt, with the sub-step */
/* offset j drawn from SplitMix64 used as a counter-based generator:    */
/* its output function at the state key + (pix + 1) * gamma, key =     */
/* seed * 2^32 + p, gamma = 0x9E3779B97F4A7C15 (the generator's golden   */
/* increment), pix = py * w + px; j is the top 24 bits as a fraction in */
/* [0, 1). Pass 0 keeps j = 1/2, the unjittered lattice.                 */
/* ------------------------------------------------------------------ */
uint64_t oracle_splitmix64_output(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

float oracle_jitter(uint32_t seed, uint32_t pass, uint64_t pix) {
    if (pass == 0) return 0.5f;
    uint64_t key = ((uint64_t)seed << 32) | pass;
    uint64_t z = oracle_splitmix64_output(key + (pix + 1) * 0x9E3779B97F4A7C15ULL);
    return (float)(z >> 40) * 0x1p-24f;
}

/* FP32 decision geometry of the ray through pixel (px, py). */
typedef struct { float o[3], d[3], t0, t1; int hit; } ray32;

static void cross_f32(const float a[3], const float b[3], float c[3]) {
    c[0] = fmaf(a[1], b[2], -(a[2] * b[1]));
    c[1] = fmaf(a[2], b[0], -(a[0] * b[2]));
    c[2] = fmaf(a[0], b[1], -(a[1] * b[0]));
}

static float dot_f32(const float a[3], const float b[3]) {
    return fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0]));
}

static void normalize_f32(float a[3]) {
    float l = sqrtf(dot_f32(a, a));
    a[0] = a[0] / l; a[1] = a[1] / l; a[2] = a[2] / l;
}

/* Pinhole camera basis (FP32, fixed order): view F = normalize(target - eye),  */
/* right R = normalize(cross(F, up)), true up U = cross(R, F).                   */
static void camera_basis32(const float *c, float F[3], float R[3], float U[3]) {
    F[0] = c[3] - c[0]; F[1] = c[4] - c[1]; F[2] = c[5] - c[2];
    normalize_f32(F);
    cross_f32(F, c + 6, R);
    normalize_f32(R);
    cross_f32(R, F, U);
}

/* Direction of the ray through pixel (px, py) of a w x h image (FP32). */
static void camera_ray32(const float *c, int w, int h, int px, int py, float d[3]) {
    float F[3], R[3], U[3];
    camera_basis32(c, F, R, U);
    float th = c[9];
    float aspect = (float)w / (float)h;
    float sxs = th * aspect;
    float qx = (float)(2 * px + 1) / (float)w;
    float qy = (float)(2 * py + 1) / (float)h;
    float sx = (qx - 1.0f) * sxs;
    float sy = (1.0f - qy) * th;
    for (int a = 0; a < 3; a++) d[a] = fmaf(sy, U[a], fmaf(sx, R[a], F[a]));
    normalize_f32(d);
}

static ray32 make_ray32(const render_job *J, int px, int py) {
    ray32 r;
    const float *c = J->cam;
    float d[3];
    camera_ray32(c, J->w, J->h, px, py, d);
    for (int a = 0; a < 3; a++) { r.o[a] = c[a]; r.d[a] = d[a]; }
    /* Sphere entry/exit through the closest point to the centre. */
    float b = dot_f32(r.o, r.d);
    float hv[3];
    for (int a = 0; a < 3; a++) hv[a] = fmaf(-b, r.d[a], r.o[a]);
    float h2 = dot_f32(hv, hv);
    float disc = J->r_out * J->r_out - h2;
    r.hit = disc > 0.0f;
    if (r.hit) {
        float sq = sqrtf(disc);
        r.t0 = fmaxf(-b - sq, 0.0f);
        r.t1 = -b + sq;
    } else {
        r.t0 = r.t1 = 0.0f;
    }
    return r;
}

/* FP64 geometry of the same ray, for the colour value (and, in the FP64-decision */
/* mode, for everything).                                                          */
typedef struct { double o[3], d[3], t0, t1; int hit; } ray64;

static ray64 make_ray64(const render_job *J, int px, int py) {
    ray64 r;
    const float *c = J->cam;
    double F[3] = {(double)c[3] - c[0], (double)c[4] - c[1], (double)c[5] - c[2]};
    double l = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    for (int a = 0; a < 3; a++) F[a] /= l;
    double up[3] = {c[6], c[7], c[8]};
    double R[3] = {F[1] * up[2] - F[2] * up[1], F[2] * up[0] - F[0] * up[2], F[0] * up[1] - F[1] * up[0]};
    l = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    for (int a = 0; a < 3; a++) R[a] /= l;
    double U[3] = {R[1] * F[2] - R[2] * F[1], R[2] * F[0] - R[0] * F[2], R[0] * F[1] - R[1] * F[0]};
    double th = c[9];
    double sx = ((2.0 * px + 1.0) / J->w - 1.0) * th * ((double)J->w / J->h);
    double sy = (1.0 - (2.0 * py + 1.0) / J->h) * th;
    double d[3];
    for (int a = 0; a < 3; a++) d[a] = F[a] + sx * R[a] + sy * U[a];
    l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; a++) { r.o[a] = c[a]; r.d[a] = d[a] / l; }
    double b = r.o[0] * r.d[0] + r.o[1] * r.d[1] + r.o[2] * r.d[2];
    double cc = r.o[0] * r.o[0] + r.o[1] * r.o[1] + r.o[2] * r.o[2] - (double)J->r_out * J->r_out;
    double disc = b * b - cc;
    r.hit = disc > 0;
    r.t0 = disc > 0 ? fmax(-b - sqrt(disc), 0.0) : 0.0;
    r.t1 = disc > 0 ? -b + sqrt(disc) : 0.0;
    return r;
}

/* FP32 trilinear interpolation of variable v at FP32 grid coordinates.   */
/* Lerps along x, then y, then z; each lerp is fmaf(f, b - a, a).          */
static inline float lerp32(float a, float b, float f) { return fmaf(f, b - a, a); }

static void grid_coord32(float p, int n, int *i0, float *f) {
    float hn = 0.5f * (float)n;
    float u = fmaf(p, hn, hn - 0.5f);
    u = fminf(fmaxf(u, 0.0f), (float)(n - 1));
    int i = (int)floorf(u);
    if (i > n - 2) i = n - 2;
    *i0 = i;
    *f = u - (float)i;
}

static float interp32_at(const float *vol, int n, int v, const int i[3], const float f[3]) {
    float c[2][2][2];
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) c[dx][dy][dz] = val(vol, n, v, i[0] + dx, i[1] + dy, i[2] + dz);
    float c00 = lerp32(c[0][0][0], c[1][0][0], f[0]);
    float c10 = lerp32(c[0][1][0], c[1][1][0], f[0]);
    float c01 = lerp32(c[0][0][1], c[1][0][1], f[0]);
    float c11 = lerp32(c[0][1][1], c[1][1][1], f[0]);
    float c0 = lerp32(c00, c10, f[1]);
    float c1 = lerp32(c01, c11, f[1]);
    return lerp32(c0, c1, f[2]);
}

static float interp32(const render_job *J, int v, const int i[3], const float f[3]) {
    return interp32_at(J->vol, J->n, v, i, f);
}

/* ------------------------------------------------------------------ */
/* Seed filtering (Section 3: only the pathlines whose seed lies in the */
/* current selection are shown). A point p (FP32 world coordinates)     */
/* passes iff it lies in the shell (FP32 |p|^2 as for a sample), passes */
/* the position brush, and every restricted variable's FP32 trilinear   */
/* value at p passes the brush: exactly the per-sample test of the ray  */
/* march. NaN coordinates fail. out[i] = 1 / 0.                          */
/* ------------------------------------------------------------------ */
void oracle_filter_points(const float *vol, int n, int nvars, float r_in, float r_out,
                          const float *lo, const float *hi, uint32_t active_mask,
                          const float *plo, const float *phi, uint32_t pmask,
                          const float *pts, int64_t npts, uint8_t *out) {
    float rin2 = r_in * r_in, rout2 = r_out * r_out;
    for (int64_t q = 0; q < npts; q++) {
        const float *p = pts + 3 * q;
        float r2 = fmaf(p[2], p[2], fmaf(p[1], p[1], p[0] * p[0]));
        int keep = (r2 >= rin2 && r2 <= rout2);
        if (keep && pmask) keep = pos_pass(p, plo, phi, pmask);
        if (keep) {
            int i0[3];
            float f[3];
            for (int a = 0; a < 3; a++) grid_coord32(p[a], n, &i0[a], &f[a]);
            for (int v = 0; v < nvars && keep; v++) {
                if (!((active_mask >> v) & 1u)) continue;
                float s = interp32_at(vol, n, v, i0, f);
                if (!(s >= lo[v] && s <= hi[v])) keep = 0;
            }
        }
        out[q] = (uint8_t)keep;
    }
}

/* FP64 trilinear interpolation at an FP64 world position (same clamping). */
static double interp64(const render_job *J, int v, const double p[3]) {
    int n = J->n, i[3];
    double f[3];
    for (int a = 0; a < 3; a++) {
        double u = (p[a] + 1.0) * 0.5 * n - 0.5;
        if (u < 0) u = 0;
        if (u > n - 1) u = n - 1;
        int k = (int)floor(u);
        if (k > n - 2) k = n - 2;
        i[a] = k;
        f[a] = u - k;
    }
    double s = 0.0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                s += w * val(J->vol, n, v, i[0] + dx, i[1] + dy, i[2] + dz);
            }
    return s;
}

static void render_pixel(const render_job *J, int px, int py, double *out, uint32_t *cnt, float *depth) {
    ray32 r = make_ray32(J, px, py);
    ray64 q = make_ray64(J, px, py);
    const float jit = oracle_jitter(J->seed, J->pass, (uint64_t)py * J->w + px);
    double C[3] = {0, 0, 0}, A = 0.0;
    uint32_t marched = 0, kept = 0;
    const double thr = 1.0 - ldexp(1.0, -12);
    float rin2 = J->r_in * J->r_in, rout2 = J->r_out * J->r_out;
    if (r.hit) {
        for (int k = 0;; k++) {
            float t = fmaf((float)k + jit, J->dt, r.t0);
            if (!(t < r.t1)) break;
            marched++;
            float p[3];
            for (int a = 0; a < 3; a++) p[a] = fmaf(t, r.d[a], r.o[a]);
            float r2 = dot_f32(p, p);
            if (!(r2 >= rin2 && r2 <= rout2)) continue;
            if (J->pmask && !pos_pass(p, J->plo, J->phi, J->pmask)) continue;
            int i0[3];
            float f[3];
            for (int a = 0; a < 3; a++) grid_coord32(p[a], J->n, &i0[a], &f[a]);
            if (J->tfvis && !J->tfvis[((size_t)(i0[2] >> 2) * J->nsb + (i0[1] >> 2)) * J->nsb + (i0[0] >> 2)])
                continue;
            int keep = 1;
            for (int v = 0; v < J->nvars && keep; v++) {
                if (!((J->active_mask >> v) & 1u)) continue;
                float s = interp32(J, v, i0, f);
                if (!(s >= J->lo[v] && s <= J->hi[v])) keep = 0;
            }
            if (!keep) continue;
            if (depth && kept == 0) *depth = t;
            kept++;
            /* Colour: FP64 value at the FP64 sample position. */
            double tk = q.t0 + ((double)k + (double)jit) * (double)J->dt;
            double p64[3];
            for (int a = 0; a < 3; a++) p64[a] = q.o[a] + tk * q.d[a];
            double vc = interp64(J, J->color_var, p64);
            double s = (vc - J->tf_lo) / ((double)J->tf_hi - J->tf_lo) * 255.0;
            if (s < 0) s = 0;
            if (s > 255) s = 255;
            int j = (int)floor(s);
            if (j > 254) j = 254;
            double w = s - j;
            double e[4];
            for (int c = 0; c < 4; c++) e[c] = J->tf[j * 4 + c] * (1.0 - w) + J->tf[(j + 1) * 4 + c] * w;
            double alpha = 1.0 - exp(-e[3] * (double)J->dt);
            double tr = 1.0 - A;
            for (int c = 0; c < 3; c++) C[c] += tr * alpha * e[c];
            A += tr * alpha;
            if (J->ert && A >= thr) break;
        }
    }
    out[0] = C[0] + (1.0 - A) * J->bg[0];
    out[1] = C[1] + (1.0 - A) * J->bg[1];
    out[2] = C[2] + (1.0 - A) * J->bg[2];
    out[3] = A + (1.0 - A) * J->bg[3];
    if (cnt) { cnt[0] = marched; cnt[1] = kept; }
    if (depth && kept == 0) *depth = INFINITY;
}

/* The same render with every decision taken in FP64 on the plain definition  */
/* (Section 2.2 restated without the method's FP32 arithmetic): the ray and    */
/* its outer-sphere interval in FP64, samples t_k = t0 + (k + 1/2) dt < t1,    */
/* p = o + t_k d, the shell test r_in^2 <= |p|^2 <= r_out^2, and the brush     */
/* test on the FP64 trilinear value at the FP64 position. Colour, transfer     */
/* function and compositing as in render_pixel. It measures how far the FP32   */
/* decisions of the method sit from the real-valued definition; it is not the  */
/* reference of the parity tests (those need the method's own decisions).     */
static void render_pixel_exact(const render_job *J, int px, int py, double *out, uint32_t *cnt) {
    ray64 q = make_ray64(J, px, py);
    double C[3] = {0, 0, 0}, A = 0.0;
    uint32_t marched = 0, kept = 0;
    const double thr = 1.0 - ldexp(1.0, -12);
    const double rin2 = (double)J->r_in * J->r_in, rout2 = (double)J->r_out * J->r_out;
    if (q.hit) {
        for (int k = 0;; k++) {
            double t = q.t0 + ((double)k + 0.5) * (double)J->dt;
            if (!(t < q.t1)) break;
            marched++;
            double p[3];
            for (int a = 0; a < 3; a++) p[a] = q.o[a] + t * q.d[a];
            double r2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
            if (!(r2 >= rin2 && r2 <= rout2)) continue;
            int keep = 1;
            for (int v = 0; v < J->nvars && keep; v++) {
                if (!((J->active_mask >> v) & 1u)) continue;
                double s = interp64(J, v, p);
                if (!(s >= (double)J->lo[v] && s <= (double)J->hi[v])) keep = 0;
            }
            if (!keep) continue;
            kept++;
            double vc = interp64(J, J->color_var, p);
            double s = (vc - J->tf_lo) / ((double)J->tf_hi - J->tf_lo) * 255.0;
            if (s < 0) s = 0;
            if (s > 255) s = 255;
            int j = (int)floor(s);
            if (j > 254) j = 254;
            double w = s - j;
            double e[4];
            for (int c = 0; c < 4; c++) e[c] = J->tf[j * 4 + c] * (1.0 - w) + J->tf[(j + 1) * 4 + c] * w;
            double alpha = 1.0 - exp(-e[3] * (double)J->dt);
            double tr = 1.0 - A;
            for (int c = 0; c < 3; c++) C[c] += tr * alpha * e[c];
            A += tr * alpha;
            if (J->ert && A >= thr) break;
        }
    }
    out[0] = C[0] + (1.0 - A) * J->bg[0];
    out[1] = C[1] + (1.0 - A) * J->bg[1];
    out[2] = C[2] + (1.0 - A) * J->bg[2];
    out[3] = A + (1.0 - A) * J->bg[3];
    if (cnt) { cnt[0] = marched; cnt[1] = kept; }
}

static void *render_worker(void *arg) {
    render_job *J = (render_job *)arg;
    const int64_t chunk = 64;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t s = J->next;
        J->next += chunk;
        pthread_mutex_unlock(&J->lock);
        if (s >= J->npix) break;
        int64_t e = s + chunk < J->npix ? s + chunk : J->npix;
        for (int64_t i = s; i < e; i++) {
            int64_t pix = J->pixels ? J->pixels[i] : i;
            int px = (int)(pix % J->w), py = (int)(pix / J->w);
            if (J->exact)
                render_pixel_exact(J, px, py, J->out + 4 * i, J->counts ? J->counts + 2 * i : NULL);
            else
                render_pixel(J, px, py, J->out + 4 * i, J->counts ? J->counts + 2 * i : NULL,
                             J->depth ? J->depth + i : NULL);
        }
    }
    return NULL;
}

/* ------------------------------------------------------------------ */
/* TF-aware skipping (a reading of the no-rebuild design of Section 2.2 */
/* applied to the transfer function). A sample contributes nothing when */
/* both TF entries it interpolates have sigma = 0: alpha is then exactly */
/* 0. The FP32 colour value of a sample in a 4^3 sub-brick lies in      */
/* [min - d, max + d] of the sub-brick's colour values (the brush       */
/* margin d; no bound when m > 2^126), and the entry index             */
/* J(v) = min(floor(clamp((v - tf_lo) * tf_scale, 0, 255)), 254), with  */
/* FP32 tf_scale = 255 / (tf_hi - tf_lo), is non-decreasing in v, so    */
/* its samples touch only entries J(min - d) .. J(max + d) + 1 -- and    */
/* entry 0 when the colour value is NaN. A sub-brick is TF-visible iff   */
/* sigma > 0 at one of those entries or at entry 0. With TF skipping,    */
/* samples in TF-invisible sub-bricks are not kept (the image is the     */
/* same; only the kept counts drop).                                     */
/* ------------------------------------------------------------------ */
static int tf_entry(float v, float tf_lo, float tf_scale) {
    float sp = (v - tf_lo) * tf_scale;
    sp = fminf(fmaxf(sp, 0.0f), 255.0f);
    int j = (int)sp;
    return j > 254 ? 254 : j;
}

void oracle_tf_visibility(const float *vol, int n, int nvars, int color_var, const float *tf,
                          float tf_lo, float tf_hi, uint8_t *vis /* nsb^3, nsb = ceil(n/4) */) {
    int nsb = (n + 3) / 4;
    size_t nsub = (size_t)nsb * nsb * nsb;
    float *mn = (float *)malloc(sizeof(float) * nsub * nvars), *mx = (float *)malloc(sizeof(float) * nsub * nvars);
    oracle_brick_minmax(vol, n, nvars, 4, mn, mx);
    float scale = 255.0f / (tf_hi - tf_lo);
    for (size_t b = 0; b < nsub; b++) {
        float lo = mn[b * nvars + color_var], hi = mx[b * nvars + color_var];
        float m = fmaxf(fabsf(lo), fabsf(hi));
        int visible = tf[3] > 0.0f || !(m <= 0x1p126f);
        if (!visible) {
            float d = fmaf(m, 0x1p-20f, 0x1p-120f);
            int j0 = tf_entry(lo - d, tf_lo, scale), j1 = tf_entry(hi + d, tf_lo, scale) + 1;
            for (int j = j0; j <= j1 && !visible; j++)
                if (tf[4 * j + 3] > 0.0f) visible = 1;
        }
        vis[b] = (uint8_t)visible;
    }
    free(mn);
    free(mx);
}

int oracle_render_pass(const float *vol, int n, int nvars, float r_in, float r_out,
                       const float *cam, int w, int h, float dt,
                       const float *lo, const float *hi, uint32_t active_mask,
                       const float *tf, int color_var, float tf_lo, float tf_hi,
                       const double *bg, int ert, const int64_t *pixels, int64_t npix,
                       double *out, uint32_t *counts, int nthreads, uint32_t seed, uint32_t pass,
                       const float *plo, const float *phi, uint32_t pmask, int tf_skip, float *depth) {
    if (n < 2 || w < 1 || h < 1 || !(dt > 0.0f)) return 1;
    render_job J;
    J.exact = 0;
    J.seed = seed; J.pass = pass;
    J.plo = plo; J.phi = phi; J.pmask = pmask;
    J.nsb = (n + 3) / 4;
    uint8_t *vis = NULL;
    if (tf_skip) {
        vis = (uint8_t *)malloc((size_t)J.nsb * J.nsb * J.nsb);
        oracle_tf_visibility(vol, n, nvars, color_var, tf, tf_lo, tf_hi, vis);
    }
    J.tfvis = vis;
    J.vol = vol; J.n = n; J.nvars = nvars; J.r_in = r_in; J.r_out = r_out;
    J.cam = cam; J.w = w; J.h = h; J.dt = dt; J.lo = lo; J.hi = hi;
    J.active_mask = active_mask; J.tf = tf; J.color_var = color_var;
    J.tf_lo = tf_lo; J.tf_hi = tf_hi; J.bg = bg; J.ert = ert;
    J.pixels = pixels; J.npix = pixels ? npix : (int64_t)w * h;
    J.out = out; J.counts = counts; J.depth = depth; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, render_worker, &J);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    free(th);
    free(vis);
    pthread_mutex_destroy(&J.lock);
    return 0;
}

int oracle_render(const float *vol, int n, int nvars, float r_in, float r_out,
                  const float *cam, int w, int h, float dt,
                  const float *lo, const float *hi, uint32_t active_mask,
                  const float *tf, int color_var, float tf_lo, float tf_hi,
                  const double *bg, int ert, const int64_t *pixels, int64_t npix,
                  double *out, uint32_t *counts, int nthreads) {
    return oracle_render_pass(vol, n, nvars, r_in, r_out, cam, w, h, dt, lo, hi, active_mask, tf, color_var,
                              tf_lo, tf_hi, bg, ert, pixels, npix, out, counts, nthreads, 0u, 0u,
                              NULL, NULL, 0u, 0, NULL);
}

/* FP64-decision render (render_pixel_exact) of all pixels or of a list. */
int oracle_render_exact(const float *vol, int n, int nvars, float r_in, float r_out,
                        const float *cam, int w, int h, float dt,
                        const float *lo, const float *hi, uint32_t active_mask,
                        const float *tf, int color_var, float tf_lo, float tf_hi,
                        const double *bg, int ert, const int64_t *pixels, int64_t npix,
                        double *out, uint32_t *counts, int nthreads) {
    if (n < 2 || w < 1 || h < 1 || !(dt > 0.0f)) return 1;
    render_job J;
    memset(&J, 0, sizeof(J));
    J.exact = 1;
    J.vol = vol; J.n = n; J.nvars = nvars; J.r_in = r_in; J.r_out = r_out;
    J.cam = cam; J.w = w; J.h = h; J.dt = dt; J.lo = lo; J.hi = hi;
    J.active_mask = active_mask; J.tf = tf; J.color_var = color_var;
    J.tf_lo = tf_lo; J.tf_hi = tf_hi; J.bg = bg; J.ert = ert;
    J.pixels = pixels; J.npix = pixels ? npix : (int64_t)w * h;
    J.out = out; J.counts = counts; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, render_worker, &J);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    return 0;
}

int oracle_num_threads(void) { return (int)sysconf(_SC_NPROCESSORS_ONLN); }

/* ------------------------------------------------------------------ */
/* Image warping (Section 2.2: frames the renderer has not finished are  */
/* interpolated by warping the last image). Source pixel s = y*w + x    */
/* with a finite depth D becomes the world point P = eye + D * d, d its  */
/* ray direction (FP32 as in the march, P by fmaf per component). P is   */
/* projected into the new camera (basis F', R', U'): v = P - eye',       */
/* z = v.F', X = v.R', Y = v.U' (FP32 fma dot products); points with     */
/* z <= 0 are dropped; qx = X / (z * (tan' * aspect)), qy = Y / (z *     */
/* tan'); target column floor((qx + 1) * (w/2)), row floor((1 - qy) *    */
/* (h/2)), dropped outside the image. Each target pixel takes the        */
/* colour of the source of smallest z, ties to the smallest source       */
/* index; pixels no source reaches take the background. With fill_holes,*/
/* a pixel no source reaches takes, among its 8 neighbours that a source */
/* reached, the one whose source has the smallest z (ties: smallest      */
/* source index), one pass over the forward result. out_src gets the     */
/* chosen source index or -1.                                            */
/* ------------------------------------------------------------------ */
void oracle_warp(const float *src_rgba, const float *src_depth, const float *cam_from, const float *cam_to,
                 int w, int h, const float *bg, int fill_holes, float *out_rgba, int32_t *out_src) {
    size_t npix = (size_t)w * h;
    float *best = (float *)malloc(sizeof(float) * npix);
    for (size_t i = 0; i < npix; i++) { best[i] = INFINITY; out_src[i] = -1; }
    float F[3], R[3], U[3];
    camera_basis32(cam_to, F, R, U);
    float aspect = (float)w / (float)h;
    float sxs = cam_to[9] * aspect, th = cam_to[9];
    float hw = (float)w * 0.5f, hh = (float)h * 0.5f;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            size_t s = (size_t)y * w + x;
            float D = src_depth[s];
            if (!(D < INFINITY)) continue;                 /* no depth (also NaN) */
            float d[3], v[3];
            camera_ray32(cam_from, w, h, x, y, d);
            for (int a = 0; a < 3; a++) v[a] = fmaf(D, d[a], cam_from[a]) - cam_to[a];
            float z = dot_f32(v, F);
            if (!(z > 0.0f)) continue;
            float X = dot_f32(v, R), Y = dot_f32(v, U);
            float qx = X / (z * sxs), qy = Y / (z * th);
            float fi = floorf((qx + 1.0f) * hw), fj = floorf((1.0f - qy) * hh);
            if (!(fi >= 0.0f && fi < (float)w && fj >= 0.0f && fj < (float)h)) continue;
            size_t t = (size_t)fj * w + (size_t)fi;
            if (z < best[t] || (z == best[t] && (int32_t)s < out_src[t])) {
                best[t] = z;
                out_src[t] = (int32_t)s;
            }
        }
    if (fill_holes) {
        int32_t *fwd = (int32_t *)malloc(sizeof(int32_t) * npix);
        memcpy(fwd, out_src, sizeof(int32_t) * npix);
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                size_t t = (size_t)y * w + x;
                if (fwd[t] >= 0) continue;
                float bz = INFINITY;
                int32_t bs = -1;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int xx = x + dx, yy = y + dy;
                        if ((dx == 0 && dy == 0) || xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                        size_t u = (size_t)yy * w + xx;
                        if (fwd[u] < 0) continue;
                        if (best[u] < bz || (best[u] == bz && fwd[u] < bs)) {
                            bz = best[u];
                            bs = fwd[u];
                        }
                    }
                out_src[t] = bs;
            }
        free(fwd);
    }
    for (size_t t = 0; t < npix; t++)
        for (int c = 0; c < 4; c++)
            out_rgba[4 * t + c] = out_src[t] >= 0 ? src_rgba[4 * (size_t)out_src[t] + c] : bg[c];
    free(best);
}
