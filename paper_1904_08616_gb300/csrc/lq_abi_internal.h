// Host-side declarations shared by the translation units of liblq.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lq.h"

namespace lq {

// A named range on the NVTX timeline around a phase of a call (shown by Nsight Systems and
// Nsight Compute; without a tool attached the calls return at once).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Geom;

// bounds-checked build: reader of one translation unit's out-of-range record (count, first
// slot); each unit registers its own at load time
using OobReaderFn = unsigned int (*)(unsigned long long* first);
void register_oob_reader(OobReaderFn r);

// per-thread error message for lq_last_error()
void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// stored sizes (bytes) of fields; 0 for invalid combinations
size_t spinor_bytes(int64_t nsites, int prec);
size_t gauge_bytes(int64_t V, int prec, int fmt);

cudaError_t convert_spinor(const Geom& g, int sp, int sl, const void* src, int dp, int dl, void* dst, cudaStream_t st,
                           int nr = 1);
// dst2 (optional): a second encoding (dp2, dfmt2, dl2) of the same links from the same pass
cudaError_t convert_gauge(const Geom& g, int sp, int sl, const void* src, int dp, int dfmt, int dl, void* dst,
                          cudaStream_t st, int dp2 = 0, int dfmt2 = 0, int dl2 = 0, void* dst2 = nullptr);

cudaError_t link_grad(const Geom& g, const void* gf, const void* psi, double scale, bool accumulate, void* out,
                      cudaStream_t st);

cudaError_t halo_pack(const Geom& g, bool dag, const void* U, const void* psi, void* to_prev, void* to_next,
                      cudaStream_t st);
cudaError_t halo_dslash(const Geom& g, double m_q, bool dag, const void* U, const void* psi, const void* from_next,
                        const void* from_prev, void* out, cudaStream_t st);

size_t cg_workspace_bytes(const Geom& g, int mode, int nrhs);
int cg_solve(const Geom& g, double m_q, int mode, int nrhs, const void* U, const void* eta, void* x,
             const lq_cg_params& prm, void* ws, size_t ws_bytes, lq_cg_info* info, cudaStream_t st);

size_t cg_workspace_bytes_schur(const Geom& g, int mode, int nrhs);
int cg_solve_schur(const Geom& g, double m_q, int mode, int nrhs, const void* U, const void* b, void* x,
                   const lq_cg_params& prm, void* ws, size_t ws_bytes, lq_cg_info* info, cudaStream_t st);

size_t cg_workspace_bytes_lattices(int n, const Geom* gs, const int* nrhs, int mode);
int cg_solve_lattices(int n, const Geom* gs, const lq_lattice* lats, int mode, const lq_cg_params& prm, void* ws,
                      size_t ws_bytes, lq_cg_info* info, cudaStream_t st);

}  // namespace lq
