/*
 * simplex.h -- C ABI of libsimplex: the block-space map H of arXiv 2208.11617
 * ("A Scalable and Energy Efficient GPU Thread Map for m-Simplex Domains"),
 * fused into per-cell kernels on dense arrays that hold a discrete orthogonal
 * m-simplex, for NVIDIA GB300 (sm_103a).
 *
 * Domain (Eq. 1, Sec. 1): Delta_n^m = { x in Z^m : x_i >= 0, x_1 + ... + x_m <= n },
 * C(n+m, m) cells.  Arrays are dense, row-major with x_m fastest, `side` cells
 * along every axis (side >= n + 1; element (x_1..x_m) at offset
 * ((x_1*side + x_2)*side + ...)*side + x_m).  Only indices <= n are ever
 * touched along the slow axes; along x_m a kernel may touch the rest of the
 * 16-byte chunk that holds index n.
 *
 * Tiles: the array is cut into tiles of block^m cells; tile X (X in Z^m) covers
 * cells block*X_i .. block*X_i + block - 1.  A CUDA block processes one tile.
 * H (Sec. 4) sends a compact grid of CUDA blocks one-to-one onto the tiles
 * that hold simplex cells; the bounding-box map f(x) = x (Sec. 2) launches all
 * N^m tiles and lets the empty ones exit.
 *
 * Conventions for every call:
 *   - return value: SIMPLEX_OK (0) or one of the error codes below; on error
 *     simplex_last_error() gives a message (thread-local), nothing is aborted
 *     and no device trap is ever raised.
 *   - device pointers are plain CUDA device addresses owned by the caller (the
 *     library never frees them); `stream` is a cudaStream_t passed as void*
 *     (NULL = legacy default stream).  Calls that take a stream are
 *     asynchronous on it unless stated otherwise.
 *   - simplex_map_t objects are owned by the library: create/destroy them in
 *     pairs.  A map is not safe for concurrent calls from several host
 *     threads.
 */
#ifndef SIMPLEX_H
#define SIMPLEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SIMPLEX_OK 0
#define SIMPLEX_EINVAL 1       /* bad argument (message says which) */
#define SIMPLEX_ENOMEM 2       /* host or device allocation failed */
#define SIMPLEX_ECUDA 3        /* a CUDA runtime or driver call failed */
#define SIMPLEX_ETIMEOUT 4     /* a bounded device-side wait gave up */
#define SIMPLEX_EUNSUPPORTED 5 /* valid request the library does not implement */

/* ---- map modes ----------------------------------------------------------- */
#define SIMPLEX_MODE_H 0  /* block-space map H (Sec. 4)                         */
#define SIMPLEX_MODE_BB 1 /* bounding box f(x) = x over N^m tiles (Sec. 2, Eq. 3)   */
#define SIMPLEX_MODE_BB_THREAD 2 /* the same bounding box with only a per-thread filter (the
                                    paper's baseline): blocks wholly outside the domain run
                                    too and their threads find no cell; identical results */

/* ---- visit-count levels ---------------------------------------------------- */
#define SIMPLEX_LEVEL_BLOCK 0
#define SIMPLEX_LEVEL_CELL 1

typedef struct simplex_map *simplex_map_t;

typedef struct simplex_map_info {
    int32_t m;              /* simplex dimension */
    int32_t r_inv;          /* 1/r, scale factor of the self-similar set (Sec. 6) */
    int32_t beta;           /* replication factor beta of the self-similar set (Sec. 6) */
    int32_t block;          /* tile side rho in cells */
    int64_t n;              /* simplex size: x_1 + ... + x_m <= n */
    int64_t side;           /* array side in cells */
    int32_t N;              /* tiles per axis of the block lattice (power of two) */
    int32_t log2N;
    int32_t band;           /* m = 2 trapezoid band height in tiles; 0 = single H2 grid */
    int32_t Ne;             /* m = 2 trapezoid form: block-triangle side (multiple of band) */
    int32_t launch;         /* automaton step form: 1 grid, 2 x-stream, 3 plane stream */
    int32_t layout;         /* m = 3, beta = 2: 0 packed grid, 1 one block range per level */
    uint64_t cells;         /* C(n+m, m), Eq. 1 */
    uint64_t useful_blocks; /* tiles holding at least one cell: C(floor(n/rho)+m, m) */
    uint64_t h_blocks;      /* CUDA blocks one H launch starts */
    uint64_t bb_blocks;     /* CUDA blocks one bounding-box launch starts (N^m) */
    uint64_t h_set_blocks;  /* blocks of the self-similar set S (Eq. generic-m) */
    uint64_t host_copy_bytes; /* bytes simplex_ca_run_host moves each way (m = 2, 3) */
    uint64_t plane_units;     /* launch 3: work units of one step in mode H (else 0) */
    uint64_t plane_units_bb;  /* launch 3: work units of one step in the bounding-box modes */
} simplex_map_info_t;

/*
 * simplex_map_create -- plan H for Delta_n^m with tile side `block`, array
 * side n + 1.
 *   m      2, 3 or 4.
 *   n      >= 0.
 *   r_inv  1/r, the scale factor of the self-similar set (Sec. 6, Eq.
 *          generic-m): 2 (r = 1/2, the paper's value) for every m, or 3 for
 *          m = 2 with beta = 3: the block triangle of side 3s is split into
 *          three squares of side s, at (0, 0), (s, 0) and (0, s), and three
 *          triangles of side s, at (2s, 0), (0, 2s) and (s, s), each split
 *          again; the lattice side is the power of three at or above
 *          ceil((n+1)/rho) and the map covers its triangle, diagonal
 *          included, with N3 (N3 + 1) / 2 blocks (band must be 0 or -1).
 *   beta   replication factor (Sec. 6).  m = 2: 2 (Eq. map2d, Thm. 1).
 *          m = 3: 2 (the packed map with the hinge of Sec. 4.3) or 3 (every
 *          corner recursed, no hinge).  m = 4: 4 (every corner recursed;
 *          Lemma 5 shows beta = 2 does not cover the 4-simplex).
 *   block  tile side rho in cells, a power of two in [4, 256].
 *   out    receives the new map.
 * Allocates host memory only.  The lattice side N is the power of two at or
 * above ceil((n+1)/rho) (n padded from above, Sec. 4.2; the bounding box uses
 * it for either r); tiles past the domain exit at once.  Errors:
 * SIMPLEX_EINVAL for a bad argument, SIMPLEX_EUNSUPPORTED for an (m, r_inv,
 * beta) the library does not map, SIMPLEX_ENOMEM.
 */
int simplex_map_create(int m, int64_t n, int r_inv, int beta, int block, simplex_map_t *out);

/* As simplex_map_create, with arrays of side `side` >= n + 1 (padding lets
 * rows start on 16-byte boundaries for any n). */
int simplex_map_create_padded(int m, int64_t n, int r_inv, int beta, int block,
                              int64_t side, simplex_map_t *out);

typedef struct simplex_map_params {
    int32_t m, r_inv, beta, block; /* as simplex_map_create */
    int64_t n;
    int64_t side;                  /* array side, >= n + 1; 0 means n + 1 */
    int32_t band;                  /* m = 2 only, see below; must be 0 or -1 for m > 2 */
    int32_t launch;                /* automaton step: 0 automatic, 1 grid, 2 x-stream, 3 plane stream (see below) */
    int32_t layout;                /* m = 3, beta = 2: 0 packed grid, 1 one range per level (see below) */
} simplex_map_params_t;

/*
 * simplex_map_create_ex -- as simplex_map_create with every planning choice
 * explicit.  For m = 2, `band` selects the form of H:
 *   band > 0 (a power of two): the trapezoid form of Sec. 4.2 (Eq. trapezoids,
 *     concurrent trapezoids), all in one launch.  The block triangle of side
 *     Ne = ceil(ceil((n+1)/block) / band) * band is cut into bands of `band`
 *     tile rows; band k is a trapezoid: a rectangle of band x (Ne - (k+1) band)
 *     tiles taken row by row, then a triangle of side `band` mapped by Eq.
 *     map2d plus its diagonal.  Ne needs no power of two, and consecutive
 *     CUDA blocks walk whole rows of tiles, which keeps stencil halos in L2.
 *   band = 0: automatic (currently 8).
 *   band = -1: the single grid of Eq. map2d (Thm. 1) on the power-of-two side
 *     N, with the diagonal row appended.
 * `launch` selects how simplex_ca_step runs the map's blocks:
 *   1 (grid): one CUDA block per block of the map, the paper's execution
 *     model (Sec. 2): the grid of a launch is the map's parallel space;
 *   2 (x-stream, m = 3 with block 32): one persistent CTA per SM takes runs
 *     of up to 16 tiles along x3 from a device work counter; the tile columns
 *     (x1, x2) of the runs are enumerated by Eq. map2d over the triangle
 *     x1 + x2 <= N - 1 (the bounding box: the N x N square).  The CTA streams
 *     each run's 32-byte-wide x-columns through a ring of TMA stages, so a
 *     column is read once per run; the map's per-tile blocks of modes H and
 *     BB become per-run work units.  The map keeps a 16-byte work counter in
 *     device memory, allocated on first use: steps of one map must not run
 *     concurrently on different streams.
 *   3 (plane stream, m = 3 with block 16 or 32; the block size does not
 *     enter the step): persistent CTAs, several per SM, take work units from
 *     a device work counter.  The tetrahedron is cut into slabs of
 *     consecutive planes x1 and each slab's cross-section x2 + x3 <= n - x1
 *     into bricks of 32 rows x2 by 128 cells x3; a unit is one brick of one
 *     slab (simplex_map_unit), numbered slab by slab so that bricks in
 *     flight are neighbours.  The CTA streams the brick along x1, staging
 *     its planes two at a time (the brick plus its one-cell halo, a box only
 *     as wide as the first plane's domain cells reach) by one TMA load into a
 *     ring of stages, and reads every staged byte once.  Slabs hold 64 planes at most and
 *     shrink towards the apex (x1 = n) to 4, so the last units of a step are
 *     short.  Mode H numbers only bricks holding cells of their slab;
 *     SIMPLEX_MODE_BB numbers every brick of the (n+1)^2 square in every slab
 *     and the empty ones are skipped by the CTA that takes them;
 *     SIMPLEX_MODE_BB_THREAD stages and computes them too, every store
 *     masked.  The same 16-byte work counter as launch 2 applies.  Plans
 *     that would need more than 320 slabs (n above about 7000) are refused
 *     with SIMPLEX_EUNSUPPORTED.
 *   0 (automatic): grid.
 * `layout` (m = 3, beta = 2 only) selects how H3 lays out its cubes:
 *   0: the single packed grid of Sec. 4.3: the big cube (N/2)^3 and one layer
 *     of height N/4 holding every smaller cube, whose blocks past the cube's
 *     side exit (about 1/8 of the blocks for large N);
 *   1: fully efficient (the alternative Sec. 4.3 closes with): every stack
 *     level b = N/4, N/8, ..., 1 gets its own range of block indices, N/(2b)
 *     cubes of b^3 blocks, in one launch: exactly (N^3 - N)/6 blocks below the
 *     plane sum = N - 1, no waste.
 * simplex_map_create and simplex_map_create_padded use band = 0, launch = 0,
 * layout = 0.
 */
int simplex_map_create_ex(const simplex_map_params_t *params, simplex_map_t *out);

/* Frees the map, its cached CUDA graphs and its capture stream.  NULL is a no-op. */
int simplex_map_destroy(simplex_map_t map);

/* Fills *out with the plan's sizes and block counts (host only). */
int simplex_map_info(simplex_map_t map, simplex_map_info_t *out);

/*
 * simplex_map_block -- host-side evaluation of the map for one CUDA block.
 * Runs the same integer decode the kernels run (H: Eq. map2d and its 3-simplex
 * and generic-m extensions; BB: f(x) = x) for linear CUDA block index `v` of a
 * launch in `mode`, and writes the tile coordinate X[0..m-1] (X[m-1] fastest)
 * to `coord`.  *valid = 1 iff that block processes a tile holding a simplex
 * cell, 0 if it exits (packing waste, overhang, or a tile past the domain).
 * v must be < h_blocks (mode H) or bb_blocks (mode BB), else SIMPLEX_EINVAL.
 * No GPU needed.
 */
int simplex_map_block(simplex_map_t map, int mode, uint64_t v, int32_t *coord, int *valid);

/*
 * simplex_map_unit -- host-side evaluation of the plane-stream work unit
 * numbering (launch 3) for unit index `w` of a step in `mode`: unit[0] = y0
 * (first row x2 of the brick, a multiple of 32), unit[1] = x0 (first cell x3,
 * a multiple of 128), unit[2] = first and unit[3] = last plane x1 the unit
 * writes.  *valid = 0 iff the unit's brick holds no cell of its slab
 * (SIMPLEX_MODE_BB; the step skips it).  The kernels run the same decode.
 * SIMPLEX_EINVAL if the map is not a plane-stream map or w is not below
 * plane_units (mode H) or plane_units_bb (the bounding-box modes).  No GPU
 * needed.
 */
int simplex_map_unit(simplex_map_t map, int mode, uint64_t w, int32_t *unit, int *valid);

/*
 * simplex_write -- coordinate-write test (Table 1 test 2 as a store-only
 * kernel): for every cell x of the domain, out[x] = splitmix32(seed ^ lin(x)),
 * lin(x) the row-major index on side n + 1 reduced mod 2^32; splitmix32 adds
 * 0x9E3779B9 and applies the MurmurHash3 32-bit finaliser.  Cells outside the
 * domain are not written.
 *   out   device, uint32, side^m elements; 16-byte aligned rows (side % 4 == 0
 *         and a 16-byte aligned base) take the 16-byte store path, anything
 *         else the 4-byte path.
 *   mode  SIMPLEX_MODE_H, SIMPLEX_MODE_BB or SIMPLEX_MODE_BB_THREAD (identical
 *         results).
 */
int simplex_write(simplex_map_t map, uint32_t *out, uint32_t seed, int mode, void *stream);

/*
 * simplex_accum -- the ACCUM test (Table 1, Sec. 5.1): every cell x of the
 * domain gets data[x] += add (mod 2^32), one read, one add and one write per
 * cell; cells outside the domain are neither read nor written.
 *   data  device, uint32, side^m elements; 16-byte aligned rows (side % 4 == 0
 *         and a 16-byte aligned base) take the 16-byte path, anything else
 *         4-byte accesses.
 *   mode  SIMPLEX_MODE_H, SIMPLEX_MODE_BB or SIMPLEX_MODE_BB_THREAD (identical
 *         results).
 * Errors: SIMPLEX_EINVAL (NULL or misaligned data, mode), SIMPLEX_ECUDA.
 */
int simplex_accum(simplex_map_t map, uint32_t *data, uint32_t add, int mode, void *stream);

/*
 * simplex_ca_init -- seeded Bernoulli state for the automaton: cell x of the
 * domain becomes 1 iff splitmix32(seed ^ lin(x)) < threshold, else 0 (p =
 * threshold / 2^32).  Cells outside the domain that share a 16-byte chunk with
 * a domain cell are written 0; others are not written.
 *   grid   device, uint8, side^m elements, m = 2 or 3, side % 16 == 0,
 *          16-byte aligned base; must be all zero outside the domain (e.g.
 *          allocated zeroed).
 *   live   device uint64 or NULL: when given, the number of live cells is
 *          ADDED to *live.
 * Uses H for its launch.  Errors: SIMPLEX_EINVAL (layout, m), SIMPLEX_ECUDA.
 */
int simplex_ca_init(simplex_map_t map, uint8_t *grid, uint32_t seed, uint32_t threshold,
                    unsigned long long *live, void *stream);

/*
 * simplex_ca_step -- one synchronous step of a life-like automaton on the
 * domain (Table 1 test 4): neighbours are the 3^m - 1 Moore offsets, a
 * neighbour outside the domain is dead, a dead cell with k live neighbours is
 * born iff bit k of `birth` is set, a live one survives iff bit k of
 * `survive` is set.  Each CUDA block stages its tile plus a one-cell halo in
 * shared memory with one TMA tiled load (out-of-range cells read as 0) and
 * writes the tile of `out` with 16-byte stores.
 *   in, out  device, uint8 (0/1), side^m elements, distinct buffers,
 *            side % 16 == 0, 16-byte aligned; both must be zero outside the
 *            domain (the step writes only 0 there).
 *   birth, survive  rule masks, bits 0..3^m-1.  B3/S23: 0x8, 0xC.
 *   live     device uint64 or NULL: the number of live cells after the step
 *            is ADDED to *live.
 *   mode     SIMPLEX_MODE_H, SIMPLEX_MODE_BB or SIMPLEX_MODE_BB_THREAD
 *            (identical results; the x-stream form runs BB_THREAD as BB).
 * m = 2 supports block 32, 64, 128; m = 3 supports block 16, 32.
 * A device-side wait that exceeds its bound is reported by a later
 * simplex_device_status() call (SIMPLEX_ETIMEOUT); the kernel never hangs.
 */
int simplex_ca_step(simplex_map_t map, const uint8_t *in, uint8_t *out, uint32_t birth,
                    uint32_t survive, unsigned long long *live, int mode, void *stream);

/*
 * simplex_ca_run -- `steps` steps a -> b -> a -> ..., as repeated
 * simplex_ca_step calls; the final state is in `a` when steps is even, in `b`
 * when odd.
 *   live       device uint64[steps + 1] or NULL.  When given, the run zeroes
 *              it, stores the live count of the initial state in live[0]
 *              and the count after step s in live[s].
 *   use_graph  nonzero: the launches are captured once into a CUDA graph
 *              (cached on the map per argument set) and replayed on `stream`.
 */
int simplex_ca_run(simplex_map_t map, uint8_t *a, uint8_t *b, int steps, uint32_t birth,
                   uint32_t survive, unsigned long long *live, int use_graph, int mode,
                   void *stream);

/*
 * simplex_ca_run_host -- end-to-end run from and to HOST memory: copies the
 * domain of host_in (side^m uint8) into device buffer a, runs simplex_ca_run
 * on the device buffers a and b, then copies the domain of the final grid
 * into host_out and the live counts into host_live (uint64[steps + 1], may be
 * NULL; needs dev_live when given).  Only the domain moves: the prefix of
 * each row that holds domain cells, in a few pitched copies per direction
 * (simplex_map_info().host_copy_bytes bytes each way: 0.55 GB instead of the
 * 1.07 GB array for m = 2, n = 32767).  Synchronises `stream` before
 * returning.  Pinned host memory gives full copy bandwidth; pageable memory
 * works but is slower.
 *   host_in   must be zero outside the domain (as every grid).
 *   host_out  domain cells receive the final state; cells outside the domain
 *             are set to 0 or left as they were.
 *   a, b      device grids, both zero outside the domain (e.g. allocated
 *             zeroed); a's domain is overwritten from host_in.
 */
int simplex_ca_run_host(simplex_map_t map, const uint8_t *host_in, uint8_t *host_out,
                        uint8_t *a, uint8_t *b, int steps, uint32_t birth, uint32_t survive,
                        unsigned long long *dev_live, unsigned long long *host_live,
                        int use_graph, int mode, void *stream);

/*
 * simplex_visit_count -- coverage check of the map (Def. 1: every simplex
 * block gets a unique CUDA block).  Launches the map in `mode` and
 * increments, with atomics:
 *   level SIMPLEX_LEVEL_BLOCK: counts[X] once per CUDA block that processes
 *     tile X; counts is uint32, dense NB^m with NB = ceil((n+1)/block).
 *   level SIMPLEX_LEVEL_CELL: counts[x] once per cell a thread processes;
 *     counts is uint32, side^m.
 * A correct map leaves 1 inside the domain and 0 outside.  counts must be
 * zeroed by the caller.
 */
int simplex_visit_count(simplex_map_t map, uint32_t *counts, int level, int mode, void *stream);

/*
 * simplex_map_test -- the MAP test of Table 1 (Sec. 5.1): the map alone.
 * Launches the map in `mode` with one CUDA block of block^m threads per block
 * of the map and one thread per cell (the paper's model of Sec. 2): the block
 * decodes its tile, each thread forms its cell coordinate x and the predicate
 * x_1 + ... + x_m <= n, and the result is consumed without touching memory
 * (the paper keeps it in a volatile variable).  The time of the call is the
 * map plus the cost of launching its blocks, the quantity the paper's 2x (m =
 * 2) and 6x (m = 3) theory is about.
 *   cells  device uint64 or NULL: when given, every block ADDS the number of
 *          its simplex cells to *cells, which must then total C(n + m, m).
 * Needs block^m <= 1024 (m = 2: block <= 32; m = 3: block <= 8; m = 4:
 * block <= 4).  Errors: SIMPLEX_EINVAL (mode, block), SIMPLEX_ECUDA.
 */
int simplex_map_test(simplex_map_t map, unsigned long long *cells, int mode, void *stream);

/*
 * simplex_edm -- the EDM test of Table 1 (Sec. 5.1) on the 2-simplex: cell
 * x = (x1, x2), x1 + x2 <= n, stands for the pair of points (i, j) =
 * (x1, n - x2) (so i <= j) and receives their Euclidean distance
 *   out[x1 * side + x2] = sqrt(sum_k (p[i][k] - p[j][k])^2)
 * in float32, summed over k = 0, 1, ... in that order with round-to-nearest
 * and no fused multiply-add, then a correctly rounded square root: the upper
 * triangle of the distance matrix of n + 1 points, diagonal (zeros) included.
 *   points  device, float32, (n + 1) x dim, row-major (point i at i * dim).
 *   dim     1 ... 16.
 *   out     device, float32, side^2 elements, 4-byte aligned (a 16-byte
 *           aligned base with side % 4 == 0 takes the 16-byte store path);
 *           cells outside the domain are not written.
 * Needs m = 2 and block 16, 32 or 64.  Errors: SIMPLEX_EINVAL, SIMPLEX_ECUDA.
 */
int simplex_edm(simplex_map_t map, const float *points, int dim, float *out, int mode, void *stream);

/* ---- batched engine ------------------------------------------------------
 *
 * Many automaton instances of uneven m and n advance together: each step is
 * ONE persistent launch over the CUDA blocks of every instance's map (H in the
 * trapezoid form for m = 2, H3 with the hinge or the generic beta = 3 cubes for
 * m = 3), cut into work items of up to 8 blocks of one instance and handed out
 * by a device-side work queue (a global atomic counter); a run of `steps`
 * steps can be captured once into a CUDA graph and replayed.  Every instance's
 * two grids, map, rule and TMA descriptors live in one caller-provided arena
 * of device memory.  Results are identical to running each instance alone
 * with simplex_ca_run.  Not part of the paper: its batched form is the
 * concurrent-kernel idea of Sec. 4.2/4.3 (several maps in flight at once)
 * carried to many independent domains.
 */
typedef struct simplex_batch *simplex_batch_t;

typedef struct simplex_instance {
    int32_t m;          /* 2 or 3 */
    int32_t block;      /* tile side: m = 2: 64 or 128; m = 3: 16 or 32 (32^3 tiles run in a second launch per
                           step), or 128: the plane stream (32 x 128 bricks streamed along x1, as launch 3 of
                           simplex_map_create_ex; all such instances run in one more launch per step) */
    int32_t beta;       /* m = 3: 2 (hinge) or 3; m = 2: 2 */
    int32_t band;       /* m = 2 trapezoid band (power of two); 0: automatic */
    int64_t n;          /* simplex size, >= 0 */
    uint32_t birth;     /* rule masks, bit k = k live neighbours */
    uint32_t survive;
    uint32_t seed;      /* initial state: Bernoulli(threshold / 2^32), as simplex_ca_init */
    uint32_t threshold;
} simplex_instance_t;

typedef struct simplex_batch_info {
    int32_t count;            /* instances */
    int32_t parity;           /* which of each instance's two grids holds its state */
    uint64_t items;           /* work items per step */
    uint64_t blocks;          /* CUDA blocks (map blocks) per step, all instances */
    uint64_t cells;           /* simplex cells, all instances */
    uint64_t arena_bytes;     /* device memory simplex_batch_bind needs */
    uint64_t grids_offset;    /* where the instances' grids start in the arena */
    uint64_t grids_bytes;     /* bytes of all grids (two per instance), from grids_offset on */
} simplex_batch_info_t;

/* Plans every instance (host memory only).  Each instance's grids have side
 * round_up(n + 1, 128).  Errors: SIMPLEX_EINVAL (an instance's parameters; the
 * message names it), SIMPLEX_ENOMEM. */
int simplex_batch_create(const simplex_instance_t *instances, int count, simplex_batch_t *out);

/* Frees the batch's host plan, its cached CUDA graphs and capture stream
 * (the bound arena stays the caller's; finish the batch's stream work
 * first).  NULL is a no-op. */
int simplex_batch_destroy(simplex_batch_t batch);

/* Sizes of the batch (host only): the fields of simplex_batch_info_t.
 * Errors: SIMPLEX_EINVAL (NULL arguments). */
int simplex_batch_info(simplex_batch_t batch, simplex_batch_info_t *out);

/* Binds the batch to `arena` (device, 256-byte aligned, >= arena_bytes,
 * owned by the caller, not shared with anything else while bound): uploads the
 * descriptors and tensor maps and zeroes every grid.  Synchronous. */
int simplex_batch_bind(simplex_batch_t batch, void *arena, uint64_t arena_bytes, void *stream);

/* Writes every instance's initial state (its seed and threshold, as
 * simplex_ca_init) into grid 0 and sets parity 0.  Asynchronous. */
int simplex_batch_init(simplex_batch_t batch, void *stream);

/*
 * simplex_batch_run -- `steps` (1..4096) steps of every instance.
 *   live  device uint64[count * (steps + 1)] or NULL: when given, it is
 *         zeroed and live[i * (steps + 1) + s] receives instance i's live
 *         cells after step s (s = 0: before the first step).
 *   use_graph  nonzero: the launches are captured once per (steps, live,
 *         parity) into a CUDA graph and replayed.
 * The state then sits in grid (parity + steps) % 2 of each instance.
 */
int simplex_batch_run(simplex_batch_t batch, int steps, unsigned long long *live, int use_graph, void *stream);

/* Device address and side of instance i's current grid (its state). */
int simplex_batch_grid(simplex_batch_t batch, int i, uint8_t **grid, int64_t *side);

/*
 * simplex_batch_run_static -- simplex_batch_run for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is a service
 * of the library, not part of the method.
 *
 * Who needs it: a host that owns every byte of device memory through its own
 * pool or budget and hands libraries fixed buffers only, or a latency-critical
 * loop that must not pay for an allocator call (cudaMalloc can synchronise
 * the device) on its hot path.  Such a caller cannot provide the arena that
 * simplex_batch_bind wants.  This entry point needs only the grids: it keeps
 * the batch's descriptors, work items, TMA maps and work-queue counters in a
 * fixed 8 MiB array of device memory compiled into the library (one per device
 * that loads the library, held until the process exits) and allocates nothing,
 * on the device or on the host.
 *
 *   grids        device, 256-byte aligned, at least grids_bytes of
 *                simplex_batch_info: both grids of every instance, laid out as
 *                in a bound arena from grids_offset on.  The instances' state
 *                is read from grid `parity` (0 or 1) and the result lands in
 *                grid (parity + steps) % 2; grids must be zero outside each
 *                domain.  The batch need not be bound.
 *   steps, live  as simplex_batch_run (live is zeroed, then filled).
 * Runs `steps` launches on `stream`.  The first call on a device looks up
 * the fixed array's address there (cudaGetSymbolAddress) and keeps it for the
 * life of the process: make that first call before any stream capture on
 * that device (this concerns the look-up only), and do not reset the device
 * (cudaDeviceReset) after it, since the array may then move.
 * Host cost: when the array does not already hold this batch's descriptors,
 * work items and tensor maps for these grids (the previous call on the device
 * was for another batch or another grids address), the call encodes the
 * tensor maps and copies all of it from ordinary (pageable) host memory, so it
 * may block the host until those copies are done; a repeated call with the
 * same batch and grids only zeroes the work-queue counters and launches.
 * Every call rewrites part of the fixed array (at least its work-queue
 * counters), so calls whose work overlaps on the GPU -- other streams, other
 * host threads -- race and give wrong results: serialise them.  A batch whose
 * descriptors, work items and counters exceed 8 MiB (about 1.2 KB per
 * instance: several thousand instances; the 2,304-instance batched workload
 * needs 2.8 MB) is rejected with SIMPLEX_EINVAL.  Batches holding plane-stream
 * instances (m = 3, block 128) are refused with SIMPLEX_EUNSUPPORTED.
 */
int simplex_batch_run_static(simplex_batch_t batch, uint8_t *grids, uint64_t grids_bytes, int parity, int steps,
                             unsigned long long *live, void *stream);

/* ---- serving with continuous batching --------------------------------------
 *
 * Jobs -- an automaton on an m-simplex of size n for a number of steps --
 * arrive over time.  The server keeps each admitted job's two grids resident
 * in a device pool capped by an HBM budget and works in rounds: one round is
 * round_steps launches of the batched persistent kernel, each advancing every
 * resident job that still has steps left by one step, whatever step each is
 * at.  Between rounds it admits
 * arrived jobs first come first served as soon as a job slot, pool memory and
 * room in the round's work list (max_items) are free, and retires finished jobs: their live count after every step and
 * a digest of their final grid are copied to host memory and their memory
 * returns to the pool.  A job's result is identical whether it runs alone or
 * among others.  Tiles of the batched passes: m = 2: 128 from n = 1024 up,
 * else 64; m = 3: 16.  With at most direct_jobs jobs resident, each job's next
 * steps (up to 4x round_steps) go out as single-instance step launches on its
 * own grids and on a side stream of its own, so light jobs run concurrently: a
 * batched pass costs more than a few jobs' own step launches.  These direct
 * launches use the tiles on which single-instance steps run fastest: m = 2:
 * 128 from n = 2560 up, else 64; m = 3: 32 from n = 352 up, else 16.
 */
typedef struct simplex_server *simplex_server_t;

typedef struct simplex_server_params {
    uint64_t hbm_budget;     /* bytes of the grid pool (both grids of every resident job) */
    int32_t max_jobs;        /* resident job slots */
    int32_t max_steps;       /* largest steps of a job (<= 4095) */
    int32_t max_items;       /* map blocks of all resident jobs together, >= 1024 (a round's
                                work items hold 1..8 blocks: fewer when the round is light) */
    int32_t max_inflight;    /* rounds the host may queue ahead of the GPU (1..64) */
    int32_t round_steps;     /* automaton steps per batched round, 1..64; 0 means 16 (a
                                direct round takes up to 4x as many, at most 64) */
    int32_t direct_jobs;     /* with at most this many resident jobs, each job's steps run as
                                single-instance step launches on a side stream of its own
                                instead of batched passes; 0 means 24, -1 never, at most 64 */
} simplex_server_params_t;

typedef struct simplex_job {
    int32_t m;               /* 2 or 3 */
    int32_t steps;           /* 1 .. max_steps */
    int64_t n;               /* >= 0 */
    uint32_t birth, survive; /* rule masks */
    uint32_t seed, threshold;/* initial state as simplex_ca_init */
} simplex_job_t;

typedef struct simplex_job_result {
    int32_t status;          /* 0 pending, 1 running, 2 done, 3 rejected (larger than the budget or a round) */
    int32_t steps;
    double arrival_ms;       /* from the trace */
    double admit_ms;         /* host time of admission */
    double done_ms;          /* device time at which its last step and its result copies had completed
                                (a CUDA event on the serving stream, against one recorded at the start) */
    uint64_t digest;         /* sum over live cells x of splitmix32(0x00D16E57 ^ lin(x)), mod 2^64 */
    uint64_t live_final;     /* live cells after the last step */
    double seen_ms;          /* host time at which the serving loop found the job complete and its
                                results became readable (simplex_server_result): done_ms plus the
                                loop's detection delay */
} simplex_job_result_t;

typedef struct simplex_server_stats {
    uint64_t submitted, completed, rejected, rounds;
    uint64_t cell_updates;   /* sum over completed work of cells x steps */
    uint64_t peak_pool_bytes;
    double wall_ms;          /* from the start of the trace to the last completion seen */
    double mean_active;      /* resident jobs per round or direct chunk launch */
    double p50_ms, p90_ms, p99_ms, max_ms, mean_ms;   /* latency: done_ms - arrival (device clock) */
    double host_issue_ms;    /* host time spent building and issuing rounds */
    double gpu_round_ms;     /* mean device time of a round: its first operation to its last */
    uint64_t launches;       /* kernels launched: admission inits, direct steps, passes, digests */
    double host_p50_ms, host_p99_ms; /* latency as the host sees it: seen_ms - arrival */
} simplex_server_stats_t;

/* Device bytes the server's arena needs for these parameters (tables + pool). */
int simplex_server_arena_bytes(const simplex_server_params_t *params, uint64_t *out);

/* Creates a server over `arena` (device, 256-byte aligned, >= the size above,
 * owned by the caller).  Allocates pinned host buffers for results. */
int simplex_server_create(const simplex_server_params_t *params, void *arena, uint64_t arena_bytes,
                          simplex_server_t *out);

/* Waits for the server's rounds and chunks still in flight, then frees its
 * streams, events and pinned host buffers (the arena stays the caller's).
 * NULL is a no-op. */
int simplex_server_destroy(simplex_server_t server);

/*
 * simplex_server_run -- serves a trace to completion (blocking).  Job i
 * arrives at arrival_s[i] seconds after the call starts (realtime != 0; with
 * realtime = 0 or arrival_s = NULL every job is available at once).  Work is
 * issued on `stream`.  Results and statistics stay queryable until the next
 * run.  A job whose grids exceed the budget, or whose work list exceeds
 * max_items, is rejected (status 3) and the others still run.  In real time
 * the calling thread polls the GPU's events while work is in flight (it
 * sleeps only when nothing is resident, until 0.2 ms before the next
 * arrival), so one host core is busy for the length of the trace.  count = 0
 * (jobs may then be NULL) runs an empty trace.  Errors: SIMPLEX_EINVAL (a
 * job's parameters, count < 0), SIMPLEX_ECUDA.
 */
int simplex_server_run(simplex_server_t server, const simplex_job_t *jobs, const double *arrival_s, int count,
                       int realtime, void *stream);

/*
 * Online use, one job at a time (single-threaded: call these from one host
 * thread).  simplex_server_begin starts a session on `stream` (the server must
 * be idle; it clears the job table and statistics).  simplex_server_submit
 * queues one job with arrival = now and returns its id (0, 1, ... in submit
 * order); it does no GPU work.  simplex_server_poll runs one turn of the
 * serving loop without waiting on the GPU: it admits queued jobs as slots and
 * pool memory allow, launches work (a direct chunk for every resident job
 * without one in flight while at most direct_jobs are resident, else a batched
 * round when fewer than max_inflight rounds are queued), and retires the
 * rounds and chunks that have completed;
 * *finished (nullable) receives how many jobs finished in that turn (done or
 * rejected).  simplex_server_wait turns the loop, waiting on the GPU when
 * nothing else can progress, until job `id` has finished, or with id < 0
 * until every submitted job has.  Results and statistics are read as after
 * simplex_server_run.  Errors: SIMPLEX_EINVAL (no session, bad job or id,
 * begin while jobs are in progress), SIMPLEX_ECUDA.  After SIMPLEX_ECUDA from
 * any serving call the server's job state is undefined: destroy it.
 */
int simplex_server_begin(simplex_server_t server, void *stream);
int simplex_server_submit(simplex_server_t server, const simplex_job_t *job, int64_t *id);
int simplex_server_poll(simplex_server_t server, int *finished);
int simplex_server_wait(simplex_server_t server, int64_t id);

/* Result of job `job` (index into the last trace or session); `live`
 * (nullable, host, steps + 1 entries) receives the live count before the
 * first and after every step. */
int simplex_server_result(simplex_server_t server, int64_t job, simplex_job_result_t *out, unsigned long long *live);

/* Statistics of the last trace or session (the fields of
 * simplex_server_stats_t): latency quantiles over the completed jobs, counts
 * of submitted, completed and rejected jobs, rounds, cell updates, launches
 * and timings.  Errors: SIMPLEX_EINVAL (NULL arguments). */
int simplex_server_stats(simplex_server_t server, simplex_server_stats_t *out);

/* The result digest of one grid: *digest += sum over live cells x of
 * splitmix32(0x00D16E57 ^ lin(x)), and *live (nullable) += the live cells.
 * Same layout rules as simplex_ca_step.  Lets a caller compare a job run alone
 * with the server's result. */
int simplex_ca_digest(simplex_map_t map, const uint8_t *grid, unsigned long long *digest, unsigned long long *live,
                      void *stream);

/*
 * simplex_device_status -- reads and clears the library's device-side error
 * word on the current device (synchronous).  *out receives 0 when no kernel
 * gave up a bounded wait since the last call; the call returns
 * SIMPLEX_ETIMEOUT if one did.
 */
int simplex_device_status(uint32_t *out);

/*
 * simplex_selftest_wait_timeout -- checks the failure-detection path of the
 * bounded device waits: launches one CTA that waits on an mbarrier nothing
 * completes, gives up after `limit_ns` (1 us .. 1 s), records the timeout in
 * the device status word and returns, leaving the context usable.  A later
 * simplex_device_status() returns SIMPLEX_ETIMEOUT (and clears it).
 * Diagnostic only; not part of any workload.
 */
int simplex_selftest_wait_timeout(uint64_t limit_ns, void *stream);

/* Message for the last failed call on this host thread ("" if none). */
const char *simplex_last_error(void);

/* Library version string. */
const char *simplex_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SIMPLEX_H */
