// Pass descriptors shared by the host planner and the pass kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"

namespace flups {

// Per-direction transform type (Section "Methodology": 4 categories; the
// symmetric ones split by face parity, Table 1; semi-unbounded by side).
enum DirType : int {
  T_PER = 0, T_UNB = 1,
  T_EE = 2, T_EO = 3, T_OE = 4, T_OO = 5,
  T_EU = 6, T_OU = 7, T_UE = 8, T_UO = 9,
};
enum Center : int { C_CELL = 0, C_NODE = 1 };

__host__ __device__ inline bool is_quarter(int t) { return t == T_EO || t == T_OE; }
__host__ __device__ inline bool is_semi(int t) { return t >= T_EU; }
__host__ __device__ inline bool is_reversed(int t) { return t == T_UE || t == T_UO; }
// coefficient taken from the real part (even at the origin face) or minus the imaginary part
__host__ __device__ inline bool is_odd_origin(int t) { return t == T_OO || t == T_OE || t == T_OU || t == T_UO; }

// Element addressing of an array seen as pencils along the pass axis:
// offset = q * ls + j * js + o * os + comp * cs, q = pencil position along the
// lane dimension (x for axis 1/2, the row y + ny z for axis 0), j = index along
// the axis, o = the remaining coordinate (blockIdx.y), comp = vector component.
struct ArrDesc {
  long long ls, js, os, cs;
};

// Green's function access in the fused pass.
struct FusedGreen {
  const void* stored;     // stored real spectrum (path precision) or nullptr for closed form
  const void* tab[3];     // closed form: per-direction |w|^2 (or FD symbol) tables, path precision
  int gext[3];            // Green index extents (x, y, z)
  int gpitch;             // x pitch of the stored spectrum (elements): gext[0] rounded up to 16 bytes
  int fold[3];            // green index = fold ? min(i, fold - i) : i, for the two non-axis dirs
  int kernel;             // closed-form kernel id (0 spectral, 2..10 HEJ order, 100 LGF2)
  double eps2_half;       // eps^2 / 2
  double scale;           // 1 / (P1 P2 P3) (closed form only; the stored spectrum is pre-scaled)
  int quarter3;           // the fused direction is a quarter-wave type
  int dims1, dims2;       // for axis-0 passes: y extent of the array (row -> (y, z))
  // Biot-Savart (spectral curl) only
  int utypes;             // transform type of each output component along the fused axis (4 bits each)
  const void* dsym[3];    // derivative symbol of extension mode kk, per direction (signed, 0 at Nyquist)
  int role[3];            // per direction: 0 r2r coefficients, 1 R2C modes, 2 C2C modes
  int quarter[3];         // per direction: quarter-wave r2r (stored m <-> extension mode 2m + 1)
  int srcodd[3];          // per direction: bit c set when component c's source type is odd at the origin
};

struct PassParams {
  const void* in;
  void* out;
  ArrDesc ai, ao;
  int axis;
  int npen;               // pencils along the lane dimension
  int W, lw, LS;          // lanes per tile (power of 2), log2, smem lane stride
  int type, center, N, n_data, P, n_modes;
  int ctypes;             // transform type of each vector component, 4 bits per component
  int n_use;              // data values used (node periodic: N)
  int ndlog;              // log2 of a power of two >= n_data, n_use, n_modes (row-mode index loops)
  int hlog;               // log2 of a power of two >= P/2 + 1
  int ct;                 // 1: compile-time tile engine (P = 2^a, W from ct_tile_width)
  int ept;                // column passes of that engine: elements per thread and stage (16 or 32)
  int rowx;               // x pass of periodic / doubled unbounded real data on the column kernels' stages
  int in_f64, out_f64;    // double-float path: the input / output is the caller's FP64 array
  int hz;                 // cell-centred doubled transform: half-zero input, half output kept (ct engine)
  int gpre;               // fused column pass: copy the tile's stored Green slice to shared memory up front
  const void* gmap;       // with gpre: two TMA tensor maps of the stored spectrum (device memory, 128-byte
                          // aligned; boxes of gbox rows and of 1 row along the fused axis), else nullptr
  int gbox;               // rows per box of the first tensor map
  int* errflag;           // device word: set to a nonzero code when a bounded wait gives up
  int dbg_wait;           // test hook: bit (code - 1) set makes the bounded wait of that code give up at once
  int rows_bulk;          // inverse row pass of complex modes: the CTA's 2W input rows arrive by one bulk
                          // copy into shared memory at byte offset rows_off (after the tile) instead of
                          // per-thread loads
  int rows_off;
  int pdl;                // launched as a programmatic dependent of the stream's previous kernel: each CTA
                          // waits for the previous grid (complete, memory visible) before touching memory
  // column passes of the compile-time engine: the input tile by TMA (0 rows: loads from registers)
  int tin_rows;           // rows along the axis copied into the tile (P/2 when pruned, else P)
  int tin_box;            // rows per TMA box
  CUtensorMap tin;        // 4D map of the input array: (x in 8-byte units, y, z, component)
  RadixPlan plan;
  const void* tw;         // exp(-2 pi i m/(2P)), m < 2P, path precision
  FusedGreen g;
};

// host launchers (passes.cu)
enum PassKind : int {
  K_FWD_REAL = 0, K_INV_REAL = 1, K_FWD_C2C = 2, K_INV_C2C = 3, K_FUSED_REAL = 4, K_FUSED_C2C = 5,
  K_CURL_REAL = 6, K_CURL_C2C = 7
};
cudaError_t launch_curl(int kind, int prec, const PassParams& p, dim3 grid, int nthreads, size_t smem, cudaStream_t st);
cudaError_t set_curl_smem_limits();
cudaError_t launch_pass(int kind, int prec, const PassParams& p, dim3 grid, int nthreads, size_t smem, cudaStream_t st);
cudaError_t set_pass_smem_limits();

// compile-time tile engine: lanes per tile for P = 2^a (32 <= P <= 2048) of a pass along `axis`
// of kind `kind`, 0 when not compiled
int ct_tile_width(int P, int prec, int axis, int kind);
// compile-time column passes of kind `kind`: elements per thread and stage (32: radix-32 stages),
// 16 otherwise
int ct_col_ept(int P, int prec, int kind);
cudaError_t launch_ct_f32(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st);
cudaError_t launch_ct_f64(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st);
cudaError_t set_limits_ct_f32();
cudaError_t set_limits_ct_f64();
cudaError_t launch_ct_df(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem, cudaStream_t st);
cudaError_t set_limits_ct_df();
cudaError_t launch_ct_df_large(int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem,
                               cudaStream_t st);
cudaError_t set_limits_ct_df_large();
// narrow compile-time tiles for small grids: lanes per tile, 0 when not compiled
int ct_small_width(int P, int prec);
cudaError_t launch_ct_small(int prec, int P, int kind, const PassParams& p, dim3 grid, int nthr, size_t smem,
                            cudaStream_t st);
cudaError_t set_limits_ct_small();

}  // namespace flups
