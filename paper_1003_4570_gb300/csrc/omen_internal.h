// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/omen.h"

struct omen_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // small device work area: reduction partials and a status word
  double* d_work = nullptr;
  size_t work_bytes = 0;
  int* d_status = nullptr;
  // Lanczos step sequences between host checks are captured once as CUDA graphs and replayed
  bool use_graphs = true;
  int reorth = OMEN_REORTH_FULL;        // full Gram–Schmidt pass policy of the Lanczos steps
  bool lock_check = true;               // single-vector lowest solves check for missed copies
  cudaStream_t cap_stream = nullptr;   // private stream the captures are recorded on
  cudaStream_t copy_stream[2] = {nullptr, nullptr};  // host<->device copies overlapped with H·X
  // device buffers of the host-buffer product, kept between calls (grown, never shrunk): a fresh
  // allocation per call costs more than the copies it serves
  void* host_scratch = nullptr;
  size_t host_scratch_bytes = 0;
  std::vector<cudaEvent_t> host_events;  // the pipeline's events, created once
};

struct omen_lattice {
  int nx, ny, nz, ncells, natoms;
  int periodic[3];
  double a_nm;
  uint8_t* d_species = nullptr;  // [natoms]
  double* d_strain = nullptr;    // [16*ncells]
  long long nbonds = 0;
};

// Launch shape of an H·X kernel: CTA width and rows per register batch (k batch: wave vectors
// per thread); zeros select the built-in defaults.
struct HxTile {
  int threads = 0, rb = 0;
};

// Per-species-pair bond blocks for the four ideal directions, at d0 (device, row-major).
struct omen_ham {
  const omen_lattice* lat = nullptr;
  int norb = 0, nspin = 1, nb = 0;        // nb = norb * nspin
  int spin_orbit = 0, precision = OMEN_F64, matrix_free = 0, bloch = 0, is_complex = 0;
  int nspecies = 1;
  long long nrows = 0;
  double eta = 2.0;
  double kvec[3] = {0, 0, 0};
  double2 phase[3];                       // exp(i k.L_d e_d) for a +1 supercell wrap along d
  // stored bond blocks in 32-slot tiles: slot (k*4+s, cell) -> p = (k*4+s)*slot_stride + cell,
  // entry e = o1*norb + o2 (A rows, B cols) at blk[((p >> 5) * norb*norb + e) * 32 + (p & 31)]
  int slot_stride = 0;                    // ncells rounded up to a multiple of 32
  double* d_blk64 = nullptr;
  float* d_blk32 = nullptr;
  float2* d_blkdf = nullptr;              // double-float (hi, lo) blocks, same tiled layout
  // matrix-free table: B0[((sa*ns + sb)*4 + k)*norb*norb + e], and the per-slot bond-length
  // factor (d0/d)^eta of the structure's strain at assembly ([16*ncells], slot layout)
  double* d_b0_64 = nullptr;
  float* d_b0_32 = nullptr;
  double* d_scale64 = nullptr;
  float* d_scale32 = nullptr;
  // onsite energies per species and orbital [ns][norb], potential per atom
  double* d_onsite = nullptr;
  float* d_onsite32 = nullptr;            // the same in FP32
  float2* d_onsite_df = nullptr;          // the same as double-float pairs (OMEN_F64_DF)
  double* d_U = nullptr;                  // [natoms]
  double lambda_so[4] = {0, 0, 0, 0};
  double* d_lambda = nullptr;             // [ns]
  HxTile tile[2];                         // H·X launch shape for FP64 [0] and FP32 [1] vectors
  HxTile ktile[2];                        // the same for the k-batched product
  // single-band effective-mass Hamiltonian on a uniform grid (lat is null; nb = 1, d_U holds
  // one potential per grid point, d_U32 its FP32 copy for FP32 vectors)
  int effmass = 0;
  int gdim[3] = {0, 0, 0};
  int gper[3] = {0, 0, 0};
  double t_hop[3] = {0, 0, 0};            // hbar^2 / (2 m0 m_d h_d^2) (eV)
  double ec = 0.0;
  float* d_U32 = nullptr;
};

// effective-mass product y = (H - sigma) x (effmass.cu)
omen_status launch_hx_effmass(omen_ctx* ctx, const omen_ham* h, const void* x, void* y, int nvec, double sigma,
                              int vec_precision, cudaStream_t st);
// U per grid point (device, eV) or null for zero; refreshes the FP32 copy
omen_status effmass_set_potential(omen_ctx* ctx, omen_ham* h, const double* U);

// status / error helpers ---------------------------------------------------------------------
omen_status set_err(omen_ctx* ctx, omen_status s, const char* fmt, ...);
#define OMEN_CUDA(ctx, call)                                                            \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return set_err(ctx, OMEN_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
  } while (0)
#define OMEN_CHECK_LAUNCH(ctx) OMEN_CUDA(ctx, cudaGetLastError())

// geometry tables (constant memory), defined in lattice.cu --------------------------------
// For A site s and direction k: the B site (4..7) of the neighbour and its cell offset.
// For B site s (0..3 = b-4) and direction k: the A site of the neighbour and its cell offset.
struct NeighbourTables {
  int a_to_b_site[4][4];
  int a_to_b_off[4][4][3];   // each component in {-1, 0}
  int b_to_a_site[4][4];
  int b_to_a_off[4][4][3];   // each component in {0, +1}
};
const NeighbourTables& host_neighbour_tables();
omen_status upload_neighbour_tables(omen_ctx* ctx);

// kernels launched from the C-ABI layer ------------------------------------------------------
omen_status launch_assemble(omen_ctx* ctx, omen_ham* ham, const omen_tb_params* p);
omen_status launch_hx(omen_ctx* ctx, const omen_ham* ham, const void* x, void* y, int nvec,
                      double sigma, int vec_precision);
omen_status launch_hx_kbatch(omen_ctx* ctx, const omen_ham* h, int nk, const double2* phases_dev, const void* x, void* y,
                             double sigma, int vec_precision);
// One structure of a multi-structure k batch: its nk wave vectors' phase table (device) and the
// element offset of its first vector in the batch's vector buffers ([nk][nrows] from there).
struct KItem {
  const omen_ham* ham;
  int nk;
  const double2* phases;
  long long x_off;
};
omen_status launch_hx_kmulti(omen_ctx* ctx, const KItem* items, int nitems, const void* x, void* y, double sigma,
                             int vec_precision);
omen_status make_phases(omen_ctx* ctx, const omen_ham* h, int nk, const double* k_host, double2** out);

// Krylov helpers (lanczos.cu)
size_t vec_elem_bytes(const omen_ham* ham, int precision);
omen_status krylov_start_from(omen_ctx* ctx, const omen_ham* ham, int prec, const void* X, int k, void* out, int nout,
                              unsigned long long seed);
