// fga_internal.h -- descriptors shared by the host layer and the sweep
// kernels of libfgadmm (not part of the public C-ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fga {

constexpr int kMaxBuckets = 24;     // distinct (type, variable-shape) groups
constexpr int kUserType0 = 64;      // first type number of a user-supplied operator (FGA_USER_TYPE0)
constexpr int kPiece = 2048;        // hub variables are reduced in pieces of this many edges
constexpr int kSmallDeg = 16;       // fast z-order: thread per variable up to this degree
constexpr int kChunkEdges = 6912;   // fast z-order: scalar edges per chunk (shared-memory buffer)
constexpr int kChunkSlots = 1024;   // fast z-order: distinct scalar variables per chunk
constexpr int kStagePairs = 128;    // fast z-order: disk pairs per bulk-copy stage
constexpr int kChunkItems = 2048;   // fast z-order: work items per chunk (upper limit)
constexpr int kLocalityBlock = 96;  // fast z-order: factors are sorted by (first, last) variable / this
// Scatter z-order: per edge one word, its scalar variable | its column << 28;
// columns 0..kColMax-1 hold a variable's first edges (in creation order),
// column kEvOverflow marks an edge of the variable's overflow row.
constexpr int kColMax = 15;
// Kernel variant ("kind"): the factor types it is compiled for (bits 0-2,
// see process_in_bucket) and the scatter order (kKindScatter).
constexpr int kKindScatter = 8;
inline __host__ __device__ constexpr int kind_types(int kind) { return kind & 7; }
inline __host__ __device__ constexpr bool kind_scatter(int kind) { return (kind & kKindScatter) != 0; }
constexpr unsigned kEvColShift = 28;
constexpr unsigned kEvVarMask = (1u << kEvColShift) - 1u;
constexpr unsigned kEvOverflow = 15u;

// Shared-memory layout of one CTA in the fast z-order (byte offsets):
// rho*m buffer (padded slot segments), z per slot, slot row starts, slot
// destinations, two bulk-copy stages of (u, x, slot/position index) for disk
// pairs, and the two stage barriers.
struct ChunkSmem {
    int pb, zl, lr, pp, st, bar, total;
    int stage_u, stage_x, stage_i, stage_bytes;   // offsets inside one stage
};
inline __host__ __device__ constexpr int align16(int v) { return (v + 15) & ~15; }
// Canonical z order: the staging rows of warp 0 (32 values plus one of pad,
// which spreads the lanes' rows over the banks), two buffers.
constexpr int kZRow = 33;
constexpr int kZShort = 8;   // canonical z: rows up to this length summed by one thread each, unstaged
inline __host__ __device__ constexpr int canonical_z_smem(int rsize) { return 2 * 32 * kZRow * rsize; }

inline __host__ __device__ constexpr ChunkSmem chunk_smem(int rsize) {
    ChunkSmem l{};
    l.pb = 0;
    l.zl = align16(l.pb + (kChunkEdges + kChunkSlots) * rsize);
    l.lr = align16(l.zl + kChunkSlots * rsize);
    l.pp = align16(l.lr + (kChunkSlots + 1) * 4);
    l.st = align16(l.pp + kChunkSlots * 4);
    l.stage_u = 0;
    l.stage_x = align16(6 * kStagePairs * rsize);
    l.stage_i = l.stage_x + align16(6 * kStagePairs * rsize);
    l.stage_bytes = l.stage_i + align16(6 * kStagePairs * 4);
    l.bar = align16(l.st + 2 * l.stage_bytes);
    l.total = l.bar + 16;
    return l;
}

// Phase-F modes: the x-update of one iteration, preceded (from the second
// iteration of a call on) by the deferred u- and n-updates of the previous
// iteration; or the u-update alone at the end of a call.  F_U_PROX_CHK is
// F_U_PROX on a check iteration (it also sums the primal residual); the
// check is a compile-time mode so that the FP64 residual arithmetic is not
// issued, predicated off, on every edge of the other iterations.
enum FMode : int { F_PROX = 0, F_U_PROX = 1, F_U_ONLY = 2, F_U_PROX_CHK = 3 };

inline __host__ __device__ constexpr bool fmode_checks(int mode) { return mode == F_U_PROX_CHK || mode == F_U_ONLY; }

// Grid-wide barrier state (device memory, zeroed before every launch):
// count and gen together are the 64-bit arrival counter of the persistent
// sweep's barrier (8-byte aligned at the start of the buffer).
struct Barrier {
    unsigned int count;
    unsigned int gen;
    int error;
    int pad;
};
static_assert(sizeof(unsigned int) * 2 == sizeof(unsigned long long), "count and gen form one 64-bit counter");

// Per-call control block written by the device.
struct Ctl {
    long long iters;   // iterations completed in this call
    double r_pri;      // RMS residuals of the last check
    double r_dual;
    int status;        // 0, or a negative FGA_E* code
    int xpar;          // x/m buffer that holds the state after the call
    int zpar;          // z buffer that holds the state after the call
    int done;          // set when the call stopped (unfused launches exit early)
    int checked;       // at least one residual check happened
    int pad;
};

// A chunk: consecutive work items of one bucket, processed by one CTA,
// whose rho*m sums are reduced per touched variable ("slot") in shared
// memory.
struct ChunkDev {
    int bucket;
    int nitems;
    long long f0;       // first work item inside the bucket
    int nslots;
    int sbase;          // first slot in slot_var / ppos
    int lrbase;         // first entry of this chunk's slot row pointers in lrow
    int pad;
};

// One bucket = all factors of one type with one variable shape.  Scalar
// edge k of factor f lives at ebase + f * arity + k (factor-major) or at
// ebase + k * nf + f (edge-major).
template <typename R>
struct BucketDev {
    int type;
    int arity;          // scalar edges per factor
    int nprm;           // parameters per factor (SoA: prm[j * nf + f])
    int per_edge;       // 1: elementwise prox, one work item per scalar edge
    int aos;            // 1: factor-major storage (ebase + f * arity + k)
    int dims[4];        // variable dimensions (types with a fixed shape)
    int nf;             // factors
    int ebase;          // first storage edge (a multiple of 4)
    int item0;          // first phase-F work item
    int nitems;         // work items (nf, or nf * arity when per_edge)
    const R *prm;       // parameters, SoA
    const R *pmat;      // MPC_DYN: projection matrices, arity x arity each
    const int *pidx;    // MPC_DYN: matrix index of each factor
};

template <typename R>
struct SweepArgs {
    int nb;
    BucketDev<R> bk[kMaxBuckets];
    int nitems_f;         // phase-F work items over all buckets
    long long E;          // scalar edges (for the RMS residuals)
    int nz;               // scalar variables

    // per-edge state, storage order
    R *x[2];
    R *m[2];              // null when m is not kept
    R *u;
    const R *rho_e;       // null: uniform rho_u
    const R *alpha_e;     // null: uniform alpha_u
    R rho_u, alpha_u;
    const int *svar;      // scalar variable of each edge
    const int *pos;       // slot of each edge in the variable-major array
    R *pvm;               // rho * m, variable-major (rows in creation order)

    // per-variable state
    R *z[2];
    const R *srho;        // sum of rho over the variable's edges
    const double *srho2;  // sum of rho^2 over the variable's edges
    const int *row;       // variable-major row pointers [nz + 1]

    // fast z-order: chunks and their per-slot partial sums
    int nchunks;
    const ChunkDev *chunks;
    const int *slot_var;          // scalar variable of every (chunk, slot)
    const int *ppos;              // position of every (chunk, slot) in part
    const int *lrow;              // per chunk: nslots + 1 offsets into the chunk buffer
    const unsigned *lidx;         // per edge: slot inside its chunk | position in the
                                  // chunk buffer (slot-sorted, padded) << 16
    R *part;                      // per-slot partial sums, variable-major
    const int *prow;              // variable-major row pointers of part [nz + 1]

    // scatter z-order (zorder 4): per edge its variable and column (ev,
    // see kEvColShift), the edge's overflow position in pos when its column
    // is kEvOverflow; pvm holds colw columns of nz values (column c of
    // variable b at c * nz + b, zero past the variable's degree) and the
    // overflow rows from ovf0 on (row pointers in prow); zovf[b] = 1 when
    // variable b has an overflow row (its z is formed by the warp items)
    const unsigned *ev;
    unsigned ovf0;
    int colw;
    const unsigned char *zovf;

    // z-update work lists
    int zorder;           // 0 canonical, 1 fast, 4 scatter
    int n_small;          // fast: variables reduced by one thread
    const int *small_vars;
    int n_witems;         // fast / scatter: warp work items (var, start, len, hub or -1)
    const int4 *witems;
    const int *hub_npieces;
    const int *hub_off;
    R *hub_part;
    unsigned int *hub_ticket;

    // three-weight mode (canonical order only; null otherwise): weight
    // class of each edge's last message (0 zero, 1 standard, 2 infinite) in
    // storage order and at the edge's variable-major position, and rho at
    // the variable-major position (null: uniform rho_u)
    unsigned char *wcls;
    unsigned char *pwcls;
    const R *prho;

    // residual partial sums, one per CTA
    double *res_pri;      // [gmax]
    double *res_dual;     // [2][gmax]
    int gmax;

    Ctl *ctl;
    Barrier *bar;
    long long k0;         // iterations done before this call
    long long K;          // iteration budget of this call
    int check_every;
    double tol_pri, tol_dual;
    long long timeout_ns;
    int skip_block;
    int xpar0, zpar0;
};

// Launchers (sweep_f32.cu / sweep_f64.cu).  `smem` = dynamic shared memory
// per CTA (the fast order's chunk buffers; 0 in canonical order).
// `kind`: 0 = every factor type, 1 = no hinge / dynamics factors.
template <typename R>
cudaError_t sweep_persistent(const SweepArgs<R> &a, int grid, int block, int smem, int kind, cudaStream_t s);
template <typename R>
cudaError_t sweep_phase_f(const SweepArgs<R> &a, int mode, int xp, int zp, int grid, int block, int smem, int kind,
                          cudaStream_t s);
template <typename R>
cudaError_t sweep_phase_z(const SweepArgs<R> &a, int zp, long long it, int chk, int grid, int block,
                          cudaStream_t s);
template <typename R>
cudaError_t sweep_check(const SweepArgs<R> &a, long long it_checked, int xp, int zp, int final_check,
                        int grid_partials, cudaStream_t s);
template <typename R>
int sweep_max_blocks_per_sm(int block, int smem, int kind);
// shard mode: this shard's running rho m sums, the rank-ordered sum of G
// shards' own sums, z from graph-wide sums (+ dual partials), and one FP64
// total of per-CTA partials
template <typename R>
cudaError_t shard_sums(const SweepArgs<R> &a, const R *s_in, R *s_out, int grid, int block, cudaStream_t s);
template <typename R>
cudaError_t shard_add_parts(const R *parts, int G, long long nz, R *total, int grid, cudaStream_t s);
template <typename R>
cudaError_t shard_z(const SweepArgs<R> &a, const R *total, int zp, int chk, int grid, int block, cudaStream_t s);
template <typename R>
cudaError_t shard_total(const double *part, int n, double *out, cudaStream_t s);

}  // namespace fga
