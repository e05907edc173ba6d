// Shared device helpers and the internal launch interface of libmsd.
// Internal to the CUDA library; nothing outside csrc/ includes it.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#define MSD_KMAX 6          // highest excitation level per spin
#define MSD_NMAX 64         // electrons per spin
#define MSD_XMAX 112        // n_h * n_p per spin (active hole x particle block)

// Row pitch (complex FP32 entries) of the mixed path's Lambda / Xi rows per
// (walker, Cholesky vector): X rounded up to 16 entries = 128 bytes, so that
// each row starts a cache line and is written in whole lines.
__host__ __device__ __forceinline__ int lam_pitch(int X) { return (X + 15) / 16 * 16; }

// Work decomposition of the per-determinant kernels: threads per block and
// strings (determinants) per thread. One block writes one partial-sum slot.
#define SE_THREADS 256
#define SE_PER_THREAD 4
#define PC_THREADS 256
#define PC_PER_THREAD 8


// ---------------------------------------------------------------- complex
__host__ __device__ __forceinline__ double2 cz(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a + b * c
__host__ __device__ __forceinline__ double2 cfma(double2 b, double2 c, double2 a) {
    return make_double2(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
// a - b * c
__host__ __device__ __forceinline__ double2 cfms(double2 b, double2 c, double2 a) {
    return make_double2(fma(-b.x, c.x, fma(b.y, c.y, a.x)), fma(-b.x, c.y, fma(-b.y, c.x, a.y)));
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    double r = b.x / b.y, d = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__host__ __device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

__host__ __device__ __forceinline__ float2 fz(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ float2 fadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 fmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 ffma(float2 b, float2 c, float2 a) {
    return make_float2(fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(b.y, c.x, a.y)));
}

// Count of kernel launches made by the library (for launch accounting).
void msd_note_launch();
// Streaming multiprocessors of the current device (queried once per device).
int msd_sm_count();

// ------------------------------------------------------------ device state
// Error word bits set by kernels (read back by the host after a call).
#define MSD_DEV_ERR_SINGULAR 1u
#define MSD_DEV_ERR_TIMEOUT  2u
#define MSD_DEV_ERR_BOUNDS   4u
// The error word is four 32-bit words: [0] the flags above, [1] unused,
// [2..3] the budget of the tensor-core kernels' pipeline waits in
// nanoseconds (one 64-bit value; about 2 s unless the caller changes it).
#define MSD_ERR_WORDS 4
#define MSD_WAIT_DEFAULT_NS 2000000000ull
// Allocate and initialise an error word on the current device (0 or -1).
int msd_err_word_alloc(unsigned** out);

// Per-spin trial tables on the device.
struct SpinTables {
    int N;              // electrons
    int nh, np;         // active holes (orbitals of D0 ever vacated) / particles
    int n_str;          // distinct excitation strings, reference string first
    int bucket[MSD_KMAX + 2];   // strings of level k: [bucket[k], bucket[k+1])
    const int* occ0;    // [N]
    const int* pos0;    // [M] position of an orbital in occ0, or -1
    const int* hole_pos;   // [nh] position in occ0 of each hole orbital
    const int* part_orb;   // [np] orbital of each particle
    const uint4* str_hp;   // [n_str] one 16-byte record per string: hole indices (0..nh-1,
                           // ascending) in bytes 0..5, particle indices (0..np-1,
                           // ascending) in bytes 8..13, so one vector load fetches both
    const int8_t* str_sign;    // [n_str] parity of the in-place -> sorted reordering
    const int* csr_off;    // [n_str+1] determinants containing each string
    const int* csr_other;  // [nnz] string of the opposite spin in that determinant
    const double* csr_c;   // [nnz] CI coefficient of that determinant
    const uint8_t* cmx;    // [sum_k k^2 n_k] x = p_i nh + h_j of entry (i, j) of each string's
                           // minor, bucket-major, a string's k^2 entries row-major (B's order)
    const uint8_t* kx;     // same layout: h_j np + p_i, the row/column of the Gram matrices
    const float* csr_cf;   // [nnz] csr_c in FP32
    long long b_off[MSD_KMAX + 2];  // per-walker offset (complex units) of each bucket's B block
    long long b_per_walker;         // sum_k b_stride(k) * (strings of level k)
    long long cmx_off[MSD_KMAX + 2];  // offset of each bucket's entries in cmx
};

// Complex entries per string in the inverse-minor arrays B: k^2 rounded up
// to even, so that in FP32 every string's block starts on a 16-byte boundary
// and two entries load as one 16-byte vector (the pad entry is zero).
__host__ __device__ __forceinline__ constexpr int b_stride(int k) { return k * k + (k & 1); }

// Hole / particle index i (< MSD_KMAX) of a string record.
__device__ __forceinline__ int rec_h(const uint4& r, int i) { return (int)(((i < 4 ? r.x : r.y) >> (8 * (i & 3))) & 0xffu); }
__device__ __forceinline__ int rec_p(const uint4& r, int i) { return (int)(((i < 4 ? r.z : r.w) >> (8 * (i & 3))) & 0xffu); }


// Pair (determinant) tables for the opposite-spin cross term.
struct PairTables {
    int n_det;
    int bucket[(MSD_KMAX + 1) * (MSD_KMAX + 1) + 1];  // by (ka, kb): index ka*(KMAX+1)+kb
    const int* a;       // [n_det] alpha string
    const int* b;       // [n_det] beta string
    const double* c;    // [n_det] coefficient
    const float* cf;    // [n_det] coefficient in FP32
    const int* det_index;  // [n_det] original position in the trial list
    // runs form of the opposite-spin term: per bucket 0 (per determinant),
    // 1 (runs sharing an alpha string) or 2 (runs sharing a beta string);
    // runs[run_off[b] ..] the first determinant of each run of bucket b
    int run_side[(MSD_KMAX + 1) * (MSD_KMAX + 1)];
    int run_off[(MSD_KMAX + 1) * (MSD_KMAX + 1) + 1];
    const int* runs;
};

// Workspace pointers for one chunk of walkers (nw walkers).
struct Work {
    int nw;             // walkers in this chunk
    int M;
    double2* Gr[2];     // [nw][N][M]     G[occ0_j][r] = Theta[r][j]
    double2* O0[2];     // [nw]           det(D0^dag phi)
    double2* Gact[2];   // [nw][nh][np]   G[h][p]
    double2* r[2];      // [nw][n_str]    ratio per string
    double2* B[2];      // [nw * b_per_walker] inverse minors (bucket-major, SoA within bucket)
    float2* Bf[2];      // FP32 copy for the mixed path (same layout)
    double2* wts[2];    // [nw][n_str]    r_s times the sum over dets containing the string of c * r_other
    double2* part;      // [nw][nslot]    per-block partial sums
    int nslot;
    unsigned* err;      // device error word
};
