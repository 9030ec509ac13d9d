/*
 * simplex_oracle.c -- CPU oracle for the discrete orthogonal m-simplex workloads.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no source with the CUDA path.
 *
 * Everything here is plain nested loops written straight from the definitions
 * in arXiv 2208.11617, so that a reader can check it against the paper by eye:
 *
 *   - Domain (Eq. 1, Sec. 1): the cells x in Z^m with x_i >= 0 and
 *     x_1 + ... + x_m <= n.  There are C(n+m, m) of them.
 *   - ACCUM-style coordinate write (Table 1 test 2, Sec. 5.1): every cell of the
 *     domain writes one value into a dense array, the rest is left untouched.
 *     The value is splitmix32(seed ^ lin(x)), lin(x) the row-major linear index
 *     on side D = n + 1 with x_m fastest, reduced mod 2^32.
 *   - Cellular automaton (Table 1 test 4, Sec. 5.1): one synchronous update of
 *     every cell of the domain from its 3^m - 1 Moore neighbours; a neighbour
 *     that is not a cell of the domain counts as dead (the paper's fixed-dead
 *     "free boundary" of its 3-simplex test, used here for every m).  The rule
 *     is a pair of bit masks: a dead cell with k live neighbours becomes alive
 *     iff bit k of `birth` is set, a live one stays alive iff bit k of
 *     `survive` is set.
 *   - Initial state: a cell of the domain is alive iff
 *     splitmix32(seed ^ lin(x)) < threshold  (Bernoulli(threshold / 2^32)).
 *   - Euclidean distance matrix (Table 1 test 3, Sec. 5.1) on the 2-simplex:
 *     cell (x1, x2) stands for the pair of points (i, j) = (x1, n - x2) and
 *     holds d(p_i, p_j), computed here in double precision from the given
 *     (float32) coordinates.
 *
 * splitmix32 is not in the paper.  It is the 32-bit golden-ratio counter step
 * (add 0x9E3779B9 = floor(2^32 / phi)) followed by the public-domain MurmurHash3
 * 32-bit finaliser (xorshift 16, multiply 0x85EBCA6B, xorshift 13, multiply
 * 0xC2B2AE35, xorshift 16), all arithmetic mod 2^32.
 *
 * Outer loops carry an OpenMP pragma so that the large cases finish in seconds;
 * each iteration of the outer loop touches disjoint output cells, so the
 * result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

uint32_t oracle_splitmix32(uint32_t z)
{
    z += 0x9E3779B9u;
    z = (z ^ (z >> 16)) * 0x85EBCA6Bu;
    z = (z ^ (z >> 13)) * 0xC2B2AE35u;
    z = z ^ (z >> 16);
    return z;
}

/* Number of threads OpenMP would use for the parallel loops (1 without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* |Delta_n^m| by enumeration (Eq. 1).  m in 1..4. */
uint64_t oracle_count_cells(int m, int64_t n)
{
    uint64_t c = 0;
    if (n < 0) return 0;
    if (m == 1) {
        for (int64_t x1 = 0; x1 <= n; x1++) c++;
    } else if (m == 2) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++) c++;
    } else if (m == 3) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++) c++;
    } else if (m == 4) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++)
                    for (int64_t x4 = 0; x1 + x2 + x3 + x4 <= n; x4++) c++;
    }
    return c;
}

/* ACCUM test (Table 1): every cell of the domain in a dense D^m uint32 array,
 * D = n + 1, receives data[x] + add (mod 2^32); the other cells are left as
 * they are.  Returns how many cells it updated. */
uint64_t oracle_accum(int m, int64_t n, uint32_t add, uint32_t *data)
{
    const int64_t D = n + 1;
    uint64_t c = 0;
    if (n < 0) return 0;
    if (m == 2) {
#pragma omp parallel for reduction(+ : c) schedule(dynamic, 8)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++) {
                data[x1 * D + x2] += add;
                c++;
            }
    } else if (m == 3) {
#pragma omp parallel for reduction(+ : c) schedule(dynamic, 1)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++) {
                    data[(x1 * D + x2) * D + x3] += add;
                    c++;
                }
    } else if (m == 4) {
#pragma omp parallel for reduction(+ : c) schedule(dynamic, 1)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++)
                    for (int64_t x4 = 0; x1 + x2 + x3 + x4 <= n; x4++) {
                        data[((x1 * D + x2) * D + x3) * D + x4] += add;
                        c++;
                    }
    }
    return c;
}

/* Coordinate-write test on a dense D^m uint32 array, D = n + 1.
 * Writes exactly the cells of the domain; returns how many it wrote. */
uint64_t oracle_write(int m, int64_t n, uint32_t seed, uint32_t *out)
{
    const int64_t D = n + 1;
    uint64_t c = 0;
    if (n < 0) return 0;
    if (m == 2) {
#pragma omp parallel for reduction(+ : c) schedule(dynamic, 8)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++) {
                int64_t lin = x1 * D + x2;
                out[lin] = oracle_splitmix32(seed ^ (uint32_t)lin);
                c++;
            }
    } else if (m == 3) {
#pragma omp parallel for reduction(+ : c) schedule(dynamic, 1)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++) {
                    int64_t lin = (x1 * D + x2) * D + x3;
                    out[lin] = oracle_splitmix32(seed ^ (uint32_t)lin);
                    c++;
                }
    } else if (m == 4) {
#pragma omp parallel for reduction(+ : c) schedule(dynamic, 1)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++)
                    for (int64_t x4 = 0; x1 + x2 + x3 + x4 <= n; x4++) {
                        int64_t lin = ((x1 * D + x2) * D + x3) * D + x4;
                        out[lin] = oracle_splitmix32(seed ^ (uint32_t)lin);
                        c++;
                    }
    }
    return c;
}

/* Seeded Bernoulli initial state on a dense D^m uint8 array (m = 2 or 3).
 * Writes every cell of the domain (0 or 1); returns the number of live cells. */
uint64_t oracle_ca_init(int m, int64_t n, uint32_t seed, uint32_t threshold, uint8_t *grid)
{
    const int64_t D = n + 1;
    uint64_t live = 0;
    if (n < 0) return 0;
    if (m == 2) {
#pragma omp parallel for reduction(+ : live) schedule(dynamic, 8)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++) {
                int64_t lin = x1 * D + x2;
                uint8_t a = oracle_splitmix32(seed ^ (uint32_t)lin) < threshold ? 1 : 0;
                grid[lin] = a;
                live += a;
            }
    } else if (m == 3) {
#pragma omp parallel for reduction(+ : live) schedule(dynamic, 1)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++) {
                    int64_t lin = (x1 * D + x2) * D + x3;
                    uint8_t a = oracle_splitmix32(seed ^ (uint32_t)lin) < threshold ? 1 : 0;
                    grid[lin] = a;
                    live += a;
                }
    }
    return live;
}

/* Is y (m coordinates) a cell of Delta_n^m?  (Eq. 1) */
static int in_domain2(int64_t y1, int64_t y2, int64_t n)
{
    return y1 >= 0 && y2 >= 0 && y1 + y2 <= n;
}

static int in_domain3(int64_t y1, int64_t y2, int64_t y3, int64_t n)
{
    return y1 >= 0 && y2 >= 0 && y3 >= 0 && y1 + y2 + y3 <= n;
}

/* One synchronous automaton step, in -> out, both dense D^m uint8 (m = 2 or 3).
 * Writes every cell of the domain in `out`; returns the number of live cells
 * after the step.  `in` is only read at cells of the domain. */
uint64_t oracle_ca_step(int m, int64_t n, uint32_t birth, uint32_t survive,
                        const uint8_t *in, uint8_t *out)
{
    const int64_t D = n + 1;
    uint64_t live = 0;
    if (n < 0) return 0;
    if (m == 2) {
#pragma omp parallel for reduction(+ : live) schedule(dynamic, 8)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++) {
                int k = 0;
                for (int d1 = -1; d1 <= 1; d1++)
                    for (int d2 = -1; d2 <= 1; d2++) {
                        if (d1 == 0 && d2 == 0) continue;
                        int64_t y1 = x1 + d1, y2 = x2 + d2;
                        if (in_domain2(y1, y2, n)) k += in[y1 * D + y2];
                    }
                uint8_t alive = in[x1 * D + x2];
                uint8_t next = alive ? (uint8_t)((survive >> k) & 1u) : (uint8_t)((birth >> k) & 1u);
                out[x1 * D + x2] = next;
                live += next;
            }
    } else if (m == 3) {
#pragma omp parallel for reduction(+ : live) schedule(dynamic, 1)
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++) {
                    int k = 0;
                    for (int d1 = -1; d1 <= 1; d1++)
                        for (int d2 = -1; d2 <= 1; d2++)
                            for (int d3 = -1; d3 <= 1; d3++) {
                                if (d1 == 0 && d2 == 0 && d3 == 0) continue;
                                int64_t y1 = x1 + d1, y2 = x2 + d2, y3 = x3 + d3;
                                if (in_domain3(y1, y2, y3, n)) k += in[(y1 * D + y2) * D + y3];
                            }
                    int64_t lin = (x1 * D + x2) * D + x3;
                    uint8_t alive = in[lin];
                    uint8_t next = alive ? (uint8_t)((survive >> k) & 1u) : (uint8_t)((birth >> k) & 1u);
                    out[lin] = next;
                    live += next;
                }
    }
    return live;
}

/* `steps` synchronous steps starting from grid a, alternating a -> b -> a ...
 * live[0] receives the live count of the initial state and live[s] the count
 * after step s.  The final state is in a when `steps` is even, else in b. */
void oracle_ca_run(int m, int64_t n, int steps, uint32_t birth, uint32_t survive,
                   uint8_t *a, uint8_t *b, uint64_t *live)
{
    const int64_t D = n + 1;
    uint64_t c = 0;
    if (m == 2) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++) c += a[x1 * D + x2];
    } else if (m == 3) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++) c += a[(x1 * D + x2) * D + x3];
    }
    live[0] = c;
    for (int s = 1; s <= steps; s++) {
        const uint8_t *src = (s % 2 == 1) ? a : b;
        uint8_t *dst = (s % 2 == 1) ? b : a;
        live[s] = oracle_ca_step(m, n, birth, survive, src, dst);
    }
}

/* Blocks of side rho (tiles of rho^m cells, block X covering cells
 * rho*X_i .. rho*X_i + rho - 1) that hold at least one cell of the domain,
 * found by visiting every cell: ind[X] = 1 for such blocks, 0 for the others.
 * ind is dense with side NB = ceil((n+1)/rho), X_m fastest.  m in 2..4. */
void oracle_block_indicator(int m, int64_t n, int rho, uint32_t *ind)
{
    const int64_t NB = (n + rho) / rho;
    if (m == 2) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                ind[(x1 / rho) * NB + x2 / rho] = 1;
    } else if (m == 3) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++)
                    ind[((x1 / rho) * NB + x2 / rho) * NB + x3 / rho] = 1;
    } else if (m == 4) {
        for (int64_t x1 = 0; x1 <= n; x1++)
            for (int64_t x2 = 0; x1 + x2 <= n; x2++)
                for (int64_t x3 = 0; x1 + x2 + x3 <= n; x3++)
                    for (int64_t x4 = 0; x1 + x2 + x3 + x4 <= n; x4++)
                        ind[(((x1 / rho) * NB + x2 / rho) * NB + x3 / rho) * NB + x4 / rho] = 1;
    }
}

/* Next state of `count` listed cells of the domain, each given by m
 * coordinates in `coords` (cell i at coords[i*m .. i*m + m - 1]), computed one
 * by one from grid `in` (dense D^m) exactly as oracle_ca_step does; out[i]
 * receives the state.  Lets a test check sampled cells of a grid too large to
 * step on the CPU as a whole. */
void oracle_ca_cells(int m, int64_t n, uint32_t birth, uint32_t survive, const uint8_t *in,
                     const int64_t *coords, int64_t count, uint8_t *out)
{
    const int64_t D = n + 1;
    for (int64_t i = 0; i < count; i++) {
        const int64_t *x = coords + i * m;
        int k = 0;
        uint8_t alive = 0;
        if (m == 2) {
            for (int d1 = -1; d1 <= 1; d1++)
                for (int d2 = -1; d2 <= 1; d2++) {
                    if (d1 == 0 && d2 == 0) continue;
                    int64_t y1 = x[0] + d1, y2 = x[1] + d2;
                    if (in_domain2(y1, y2, n)) k += in[y1 * D + y2];
                }
            alive = in[x[0] * D + x[1]];
        } else if (m == 3) {
            for (int d1 = -1; d1 <= 1; d1++)
                for (int d2 = -1; d2 <= 1; d2++)
                    for (int d3 = -1; d3 <= 1; d3++) {
                        if (d1 == 0 && d2 == 0 && d3 == 0) continue;
                        int64_t y1 = x[0] + d1, y2 = x[1] + d2, y3 = x[2] + d3;
                        if (in_domain3(y1, y2, y3, n)) k += in[(y1 * D + y2) * D + y3];
                    }
            alive = in[(x[0] * D + x[1]) * D + x[2]];
        }
        out[i] = alive ? (uint8_t)((survive >> k) & 1u) : (uint8_t)((birth >> k) & 1u);
    }
}

/* Euclidean distance matrix on the 2-simplex (Table 1 test 3): out (dense
 * D x D, D = n + 1, double) receives at (x1, x2), x1 + x2 <= n, the distance
 * between points i = x1 and j = n - x2 of `points` ((n + 1) x dim, row-major,
 * float32), in double precision; other entries are left untouched. */
void oracle_edm(int64_t n, int dim, const float *points, double *out)
{
    const int64_t D = n + 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t x1 = 0; x1 <= n; x1++)
        for (int64_t x2 = 0; x1 + x2 <= n; x2++) {
            const float *a = points + x1 * dim, *b = points + (n - x2) * dim;
            double s = 0.0;
            for (int k = 0; k < dim; k++) {
                const double d = (double)a[k] - (double)b[k];
                s += d * d;
            }
            out[x1 * D + x2] = sqrt(s);
        }
}

/* The distances of `count` listed cells (x1, x2) of the 2-simplex (coords[2i],
 * coords[2i + 1]), one by one, as oracle_edm defines them: checks sampled cells
 * of a matrix too large for the CPU to fill as a whole. */
void oracle_edm_cells(int64_t n, int dim, const float *points, const int64_t *coords, int64_t count, double *out)
{
    for (int64_t i = 0; i < count; i++) {
        const int64_t x1 = coords[2 * i], x2 = coords[2 * i + 1];
        const float *a = points + x1 * dim, *b = points + (n - x2) * dim;
        double s = 0.0;
        for (int k = 0; k < dim; k++) {
            const double d = (double)a[k] - (double)b[k];
            s += d * d;
        }
        out[i] = sqrt(s);
    }
}
