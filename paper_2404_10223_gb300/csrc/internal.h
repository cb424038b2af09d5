// Internal declarations shared by the host planner, the kernels and the ABI layer.
#pragma once
#include <cuda_bf16.h>
#include <vector_types.h>

#include <cstdint>
#include <string>
#include <vector>

#ifdef __CUDACC__
#define TNQE_HD __host__ __device__
#else
#define TNQE_HD
#endif

namespace tnqe {

// A particle-number charge (n_alpha, n_beta) is coded as n_alpha * 16 + n_beta.
constexpr int QSTRIDE = 16;
constexpr int QSPACE = 256;
constexpr int MAXSEC = 160;            // sectors per bond
TNQE_HD inline int local_charge(int k) { return (k & 1) * QSTRIDE + (k >> 1); }

struct SectorTable {                   // one bond: sectors in ascending charge
  int nsec;
  int q[MAXSEC];
  int off[MAXSEC];
  int dim[MAXSEC];
};

// ----------------------------------------------------------------------------- host planning
struct Gate {
  int site;        // acts on sites (site, site+1)
  int side;        // 0: singular values join the left tensor, 1: the right tensor
  double c, s;     // rotation J = [[c, -s], [s, c]] at rows/columns (site, site+1)
};

struct GivensPlan {
  std::vector<Gate> gates;   // in application order
  int neg_site;              // site whose orbital flips sign (det V = -1), else -1
};

GivensPlan givens_plan(const double* V, int N);
void gate_matrix(double c, double s, double* G16x16);   // row (k1',k2'), col (k1,k2), K = 4 k1 + k2
void rotate_integrals(const double* h1, const double* eri, const double* U, int N,
                      std::vector<double>& h_out, std::vector<double>& eri_out);

struct MpoSite {            // stage-2 operator of one site as CSR over output rows
  int Din, Dout;            // channels at bond t and t+1
  std::vector<int> rowptr;  // size 4*Dout + 1, row = k * Dout + w'
  std::vector<int> col;     // w * 4 + k'
  std::vector<double> val;
};
struct Mpo {
  std::vector<int> dims;    // N + 1 channel counts; channel 0 = identity string, 1 = completed H
  std::vector<MpoSite> sites;
};
Mpo build_mpo(const double* h1, const double* eri, int N);

// ----------------------------------------------------------------------------- device descriptors
struct RotDesc {
  int N, chi_rot, ngates, neg_site, renorm, max_sweeps;
  int pad_out, pad_;              // pad_out: leave every site as [cap_l][4][cap_r], zero-filled
  double cutoff;
  const double* src;              // input MPS j
  const long long* src_off;       // N site offsets into src
  const int* src_dims;            // N + 1
  const SectorTable* src_sec;     // N + 1
  double* work;                   // rotated MPS, per-site capacity
  const long long* work_off;      // N site offsets into work
  int* work_dims;                 // N + 1
  const int* work_cap;            // N + 1 bond capacities
  SectorTable* work_sec;          // N + 1
  const double* gates;            // ngates * 256
  const int* gate_site;
  const int* gate_side;
  double* theta;                  // scratch: two-site tensor
  double* bbuf;                   // SVD blocks (scaled copies of the gated two-site blocks)
  double* wbuf;                   // B V per block
  double* qbuf;                   // V per block
  double* tbuf;                   // n x n temporaries per block
  float* w32;                     // FP32 working copy of each block
  float* q32;                     // FP32 rotations of each block
  int* meta;                      // scratch ints
  long long meta_cap;
  double* discarded;
  int* status;
  double* flops;                  // algorithmic FLOPs of this rotation (written at exit)
};

struct GemmDesc {                 // C[M x N] = op(A) * B ; all row-major
  int M, N, K, transA;            // transA: A stored K x M
  int lda, ldb, ldc, pad;
  const double* A;
  const double* B;
  double* C;
};

struct SpmmDesc {                 // Y[a][row][:] = sum val * X[a][col][:], rows = 4*Dout (k*Dout + w')
  int chi_a, nrows, ncols_x, width;  // width = ket bond dim (b')
  const int* rowptr;
  const int* col;
  const double* val;
  const double* X;                // [a][4*Din][width]
  double* Y;                      // [a][4][Dout][width] == [a][nrows][width]
};

// split-precision contraction (kernels_tc.cu)
struct PackDesc {                 // mode 0: ketT[(k',b')][b] = B[b][k'][b'];  mode 1: braT[a'][(a,k)] = A[a][k][a']
  const double* src;
  float* dst;
  int cl, cr, ld, mode;
};
struct SpmmTDesc {                // Yt[(w',b')][(a,k)] = sum W[(w',k),(w,k')] X[(a,w)][(k',b')]
  const int* rowptr;
  const int* col;
  const float* val;
  const float* X;
  float* Yt;
  int chi_a, Din, Dout, width, ldy, pad;
};
struct TcGemmDesc;

// sliced-BF16 contraction (kernels_oz.cu); double-floats are float2 (hi, lo)
struct SliceRowsDesc {            // rows of src (K values, stride ld) -> dst[s * slice_stride + r * ldK + k]
  const float2* src;
  __nv_bfloat16* dst;
  int* exps;
  long long ld, ldK, slice_stride;
  int K, ns;
};
struct SliceColsDesc {            // columns of src[K][ncols] (row stride ld) -> K-major slices per column
  const float2* src;
  __nv_bfloat16* dst;
  int* exps;
  long long ld, ldK, slice_stride;
  int K, ncols, ns, pad;
};
struct SliceSiteDesc {            // FP64 site tensor [cl][4][cr] -> K-major slices (mode 0 ket, 1 bra)
  const double* src;
  __nv_bfloat16* dst;
  int* exps;
  long long ldK, slice_stride;
  int cl, cr, mode, ns;
};
struct SpmmDfDesc {               // Y[a][row][:] = sum val * X[a][col][:] in double-float
  int chi_a, nrows, ncols_x, width;
  const int* rowptr;
  const int* rowperm;             // rows by descending nonzero count
  const int* col;
  const float2* val;
  const float4* ent;              // per nonzero: (value hi, value lo, column as int bits, 0)
  const float2* X;
  float2* Y;
};
struct OzGemmDesc;

// block-sparse FP64 contraction (kernels_block.cu).  Every bond index carries a
// particle-number charge and every MPO channel the charge change of the operator
// string it carries, so L[a][w][b] can be nonzero only when q(a) = q(b) + d(w),
// and X, Y likewise.  Only those blocks are computed and read; the arrays keep
// the dense capacity layout of the dense form ([a][w][b], [a][w][k'][b'],
// [a][k][w'][b']), so the contraction can be planned before the rotation has
// decided the ket's sector dimensions.
struct BsChannels {               // channels of one MPO bond grouped by charge change d(w)
  int ncls, pad_;
  const int* off;                 // ncls + 1 offsets into w
  const int* d;                   // 2 ncls: (d_alpha, d_beta) of each class
  const int* w;                   // the channel ids, class by class
};
struct BsRows {                   // rows k * Dout + w' of one MPO site grouped by d(w') - q(k)
  int ncls, pad_;
  const int* off;                 // ncls + 1 offsets into rows
  const int* d;                   // 2 ncls
  const int* rows;                // class by class, rows by descending nonzero count
  const int* nnz;                 // ncls: nonzeros of each class
};
struct BsSiteDesc {               // one (pair, site)
  int Din, Dout, ca, ca2;         // MPO bond dims; bra bond dims
  int capb, capb2, pad0, pad1;    // ket layout strides (capacities)
  const double* A;                // bra site [ca][4][ca2]
  const double* B;                // ket site [capb][4][capb2]
  const SectorTable* braL;        // bra bonds t, t + 1
  const SectorTable* braR;
  const SectorTable* ketL;        // ket bonds t, t + 1 (written by the rotation for rotated kets)
  const SectorTable* ketR;
  const double* Lin;              // [ca][Din][capb]
  double* Lout;                   // [ca2][Dout][capb2]
  double* X;                      // [ca][Din][4][capb2]
  double* Y;                      // [ca][4][Dout][capb2]
  const int* rowptr;              // MPO site CSR (rows k * Dout + w', columns w * 4 + k')
  const int* col;
  const double* val;
  BsChannels chL, chR;            // channel classes of bonds t and t + 1
  BsRows rows;                    // row classes of site t
};
constexpr int BS_MAXRC = 128;      // row classes per MPO site

// status bits written by kernels
constexpr int STATUS_NOCONV = 1;
constexpr int STATUS_OVERFLOW = 2;

// kernel launchers (kernels_*.cu); return cudaError_t as int
int launch_rotate(const RotDesc* d_descs, int npairs, int smem_bytes, void* stream);
int launch_gemm_f64(const GemmDesc* d_descs, const long long* d_tile_prefix, int nprob,
                    long long total_tiles, void* stream);
int launch_spmm_f64(const SpmmDesc* d_descs, const long long* d_row_prefix, int nprob,
                    long long total_rows, void* stream);
int launch_extract(const double* const* d_final, int npairs, double* H, double* S, void* stream);
int launch_pack_sites(const PackDesc* d, const long long* prefix, int n, long long total, void* stream);
int launch_gemm_tf32x3(const TcGemmDesc* d, const long long* tile_prefix, int nprob, long long total_tiles,
                       long long max_spin, int* err, void* stream);
int launch_spmm_t_f32(const SpmmTDesc* d, const long long* prefix, int nprob, long long total, void* stream);
int launch_extract_f32(const float* const* fin, int npairs, int ld, double* H, double* S, void* stream);
int launch_slice_rows(const SliceRowsDesc* d, const long long* prefix, int n, long long rows, void* stream);
int launch_slice_cols(const SliceColsDesc* d, const long long* prefix, int n, long long blocks, int max_k,
                      void* stream);
int launch_slice_sites(const SliceSiteDesc* d, const long long* prefix, int n, long long rows, void* stream);
int launch_spmm_df(const SpmmDfDesc* d, const long long* prefix, int n, long long total, void* stream);
// shared-memory form: one CTA per (problem, a, bw ket columns); prefix counts CTAs
int spmm_df_smem_width(int max_ncols_x);   // bw in {8, 4, 2, 1}, 0 if the X slab does not fit
int launch_spmm_df_smem(const SpmmDfDesc* d, const long long* prefix, int n, long long blocks, int bw,
                        int max_ncols_x, void* stream);
int launch_unit_env(float2* const* env, int n, void* stream);
int launch_scatter_pairs(const double* h, const double* s, const int* idx, int n, double* H, double* S,
                         void* stream);
int launch_unit_env_f64(double* const* env, int n, void* stream);
int launch_unit_env_f32(float* const* env, int n, void* stream);
int launch_extract_df(const float2* const* fin, int npairs, double* H, double* S, void* stream);
int launch_gemm_bf16s(const OzGemmDesc* d, const long long* tile_prefix, int nprob, long long total_tiles,
                      long long max_spin, int* err, int bn, int ns, void* stream);
// block-sparse FP64 stages; prefix[p] counts the CTAs of the descriptors before p;
// flops (device, 3 doubles) accumulates the algorithmic FLOPs of stages 1, 2, 3;
// threads: CTA size, 64, 128 or 256
int launch_bs_stage1(const BsSiteDesc* d, const long long* prefix, int n, long long total, double* flops,
                     int threads, void* stream);
int launch_bs_stage2(const BsSiteDesc* d, const long long* prefix, int n, long long total, double* flops,
                     int threads, void* stream);
int launch_bs_stage3(const BsSiteDesc* d, const long long* prefix, int n, long long total, double* flops,
                     int threads, void* stream);
int launch_dependence(const double* d_S, int M, double eps, int max_sweeps, double* d_resid, int* d_status,
                      void* stream);
int launch_solve(const double* d_H, const double* d_S, int M, double eps, int max_sweeps,
                 double* d_E, double* d_C, int* d_rank, double* d_kappa, int* d_status, void* stream);

}  // namespace tnqe
