// extern "C" entry points of liblq (declared in include/lq.h): argument checks, then
// dispatch to the kernels.  Nothing is launched when a check fails.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "lq_abi_internal.h"
#include "dslash_dispatch.cuh"

namespace lq {

thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int fail(int status, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(LQ_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

size_t spinor_bytes(int64_t nsites, int prec) {
    switch (prec) {
        case LQ_F64:
        case LQ_F64X: return (size_t)nsites * 192;
        case LQ_F32: return (size_t)nsites * 96;
        case LQ_F16S: return (size_t)nsites * 52;
        case LQ_I32S: return (size_t)nsites * 100;
        default: return 0;
    }
}

// readers of the per-translation-unit out-of-range records of the bounds-checked build
static std::vector<OobReaderFn>& oob_readers() {
    static std::vector<OobReaderFn> v;
    return v;
}
void register_oob_reader(OobReaderFn r) { oob_readers().push_back(r); }

size_t gauge_bytes(int64_t V, int prec, int fmt) {
    if (fmt != 18 && fmt != 12 && fmt != 10) return 0;
    switch (prec) {
        case LQ_F64:
        case LQ_F64X: return (size_t)V * 4 * fmt * 8;
        case LQ_F32:
        case LQ_I32S: return (size_t)V * 4 * fmt * 4;
        case LQ_F16S: return (size_t)V * 4 * fmt * 2;
        default: return 0;
    }
}

}  // namespace lq

using namespace lq;

namespace {

// site-fields per call: every 32-bit slot index of a multi-field spinor (at most 12 per
// site-field) stays below 2^32
constexpr int64_t kMaxSiteFields = int64_t(1) << 28;

bool valid_prec(int p) { return p == LQ_F64 || p == LQ_F32 || p == LQ_F16S || p == LQ_F64X || p == LQ_I32S; }
bool valid_layout(int l) { return l == LQ_LAYOUT_LEX || l == LQ_LAYOUT_EO; }
bool valid_fmt(int f) { return f == LQ_LINK18 || f == LQ_LINK12 || f == LQ_LINK10; }
bool valid_cg_mode(int m) {
    return m == LQ_CG_F64 || m == LQ_CG_MIXED_F32 || m == LQ_CG_MIXED_F16 || m == LQ_CG_F64X || m == LQ_CG_MIXED_I32;
}
bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

int check_dims(const int32_t* dims, Geom* g) {
    if (!dims) return fail(LQ_ERR_ARG, "dims is NULL");
    long long v = 1;
    for (int i = 0; i < 4; ++i) {
        if (dims[i] < 2 || (dims[i] & 1))
            return fail(LQ_ERR_DIMS, "lattice extent %d is %d: extents must be even and >= 2", i, (int)dims[i]);
        v *= dims[i];
        if (v > 100000000LL) return fail(LQ_ERR_DIMS, "lattice volume exceeds 10^8 sites");
    }
    *g = make_geom(dims);
    return LQ_OK;
}

// a t-slab of a decomposed lattice: x, y, z even >= 2, Lt_local >= 1
int check_slab(const int32_t* dims, Geom* g) {
    if (!dims) return fail(LQ_ERR_ARG, "dims is NULL");
    long long v = 1;
    for (int i = 0; i < 4; ++i) {
        const bool ok = (i < 3) ? (dims[i] >= 2 && !(dims[i] & 1)) : (dims[i] >= 1);
        if (!ok) return fail(LQ_ERR_DIMS, "slab extent %d is %d: x, y, z even and >= 2, t >= 1", i, (int)dims[i]);
        v *= dims[i];
        if (v > 100000000LL) return fail(LQ_ERR_DIMS, "slab volume exceeds 10^8 sites");
    }
    *g = make_geom(dims);
    return LQ_OK;
}

int check_ptr(const void* p, const char* name) {
    if (!p) return fail(LQ_ERR_ARG, "%s is NULL", name);
    if (!aligned16(p)) return fail(LQ_ERR_ALIGN, "%s is not 16-byte aligned", name);
    return LQ_OK;
}

int do_apply(const int32_t dims[4], double m_q, int32_t prec, int32_t fmt, int32_t layout, const void* U,
             const void* psi, void* out, void* stream, bool dag, int32_t nrhs = 1) {
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (nrhs < 1 || (int64_t)nrhs * g.V > kMaxSiteFields)
        return fail(LQ_ERR_ARG, "nrhs must be >= 1 with nrhs * V <= 2^28");
    if (layout == LQ_LAYOUT_EO && (nrhs & (nrhs - 1)) != 0)
        return fail(LQ_ERR_ARG, "EO fields interleave a power-of-two number of right-hand sides (got %d)", (int)nrhs);
    if (nrhs > 32 && layout == LQ_LAYOUT_EO) return fail(LQ_ERR_ARG, "at most 32 interleaved right-hand sides");
    if (!valid_prec(prec)) return fail(LQ_ERR_ARG, "bad precision %d", (int)prec);
    if (!valid_fmt(fmt)) return fail(LQ_ERR_ARG, "bad link format %d", (int)fmt);
    if (!valid_layout(layout)) return fail(LQ_ERR_ARG, "bad layout %d", (int)layout);
    if (prec == LQ_F64X && fmt != LQ_LINK18) return fail(LQ_ERR_ARG, "LQ_F64X fields use 18-real links");
    if (!isfinite(m_q)) return fail(LQ_ERR_ARG, "m_q is not finite");
    if ((r = check_ptr(U, "U")) || (r = check_ptr(psi, "psi")) || (r = check_ptr(out, "out"))) return r;
    const size_t sb = spinor_bytes((int64_t)g.V * nrhs, prec), gb = gauge_bytes(g.V, prec, fmt);
    if (overlap(out, sb, psi, sb) || overlap(out, sb, U, gb))
        return fail(LQ_ERR_ALIGN, "out overlaps psi or U");
    cudaStream_t st = (cudaStream_t)stream;
    // LEX fields are stacked: any count splits into power-of-two groups of consecutive
    // fields; EO fields are interleaved and go in one launch
    const size_t field = spinor_bytes(g.V, prec);
    for (int first = 0; first < nrhs;) {
        int lnr = 0;
        if (layout == LQ_LAYOUT_EO) {
            while ((1 << (lnr + 1)) <= nrhs) ++lnr;
        } else {
            while ((1 << (lnr + 1)) <= nrhs - first && lnr < 5) ++lnr;
        }
        // scaled stacked fields keep each field's scales after its elements; batch them one by one
        if ((prec == LQ_F16S || prec == LQ_I32S) && layout == LQ_LAYOUT_LEX) lnr = 0;
        const void* pin = (const char*)psi + (layout == LQ_LAYOUT_LEX ? field * first : 0);
        void* pout = (char*)out + (layout == LQ_LAYOUT_LEX ? field * first : 0);
        cudaError_t e;
        if (prec == LQ_F64) e = apply_f64(g, m_q, fmt, layout, dag, U, pin, pout, st, lnr);
        else if (prec == LQ_F64X) e = apply_f64x(g, m_q, fmt, layout, dag, U, pin, pout, st, lnr);
        else if (prec == LQ_F32) e = apply_f32(g, m_q, fmt, layout, dag, U, pin, pout, st, lnr);
        else if (prec == LQ_I32S) e = apply_i32(g, m_q, fmt, layout, dag, U, pin, pout, st, lnr);
        else e = apply_f16(g, m_q, fmt, layout, dag, U, pin, pout, st, lnr);
        if (e != cudaSuccess) return cuda_fail(e, dag ? "dslash_adjoint launch" : "dslash_apply launch");
        first += 1 << lnr;
    }
    return LQ_OK;
}

}  // namespace

extern "C" {

size_t lq_field_bytes(const int32_t dims[4], int32_t kind, int32_t prec, int32_t link_fmt, int32_t layout) {
    Geom g;
    if (check_dims(dims, &g) != LQ_OK || !valid_prec(prec) || !valid_layout(layout)) return 0;
    if (kind == LQ_FIELD_SPINOR) return spinor_bytes(g.V, prec);
    if (kind == LQ_FIELD_GAUGE) return valid_fmt(link_fmt) ? gauge_bytes(g.V, prec, link_fmt) : 0;
    return 0;
}

int lq_dslash_apply(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt, int32_t layout,
                    const void* U, const void* psi, void* out, void* cuda_stream) {
    NvtxRange nvtx("lq_dslash_apply");
    return do_apply(dims, m_q, prec, link_fmt, layout, U, psi, out, cuda_stream, false);
}

int lq_dslash_adjoint(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt, int32_t layout,
                      const void* U, const void* psi, void* out, void* cuda_stream) {
    NvtxRange nvtx("lq_dslash_adjoint");
    return do_apply(dims, m_q, prec, link_fmt, layout, U, psi, out, cuda_stream, true);
}

int lq_dslash_apply_multi(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt, int32_t layout,
                          int32_t nrhs, const void* U, const void* psi, void* out, void* cuda_stream) {
    NvtxRange nvtx("lq_dslash_apply_multi");
    return do_apply(dims, m_q, prec, link_fmt, layout, U, psi, out, cuda_stream, false, nrhs);
}

int lq_dslash_adjoint_multi(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt, int32_t layout,
                            int32_t nrhs, const void* U, const void* psi, void* out, void* cuda_stream) {
    NvtxRange nvtx("lq_dslash_adjoint_multi");
    return do_apply(dims, m_q, prec, link_fmt, layout, U, psi, out, cuda_stream, true, nrhs);
}

int lq_dslash_hop(const int32_t dims[4], int32_t out_parity, int32_t dagger, double a, double b, int32_t prec,
                  int32_t link_fmt, const void* U, const void* psi_other, const void* y, void* out,
                  void* cuda_stream) {
    NvtxRange nvtx("lq_dslash_hop");
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (out_parity != 0 && out_parity != 1) return fail(LQ_ERR_ARG, "out_parity must be 0 or 1");
    if (!valid_prec(prec)) return fail(LQ_ERR_ARG, "bad precision %d", (int)prec);
    if (!valid_fmt(link_fmt)) return fail(LQ_ERR_ARG, "bad link format %d", (int)link_fmt);
    if (prec == LQ_F64X && link_fmt != LQ_LINK18) return fail(LQ_ERR_ARG, "LQ_F64X fields use 18-real links");
    if (!isfinite(a) || !isfinite(b)) return fail(LQ_ERR_ARG, "a and b must be finite");
    if ((r = check_ptr(U, "U")) || (r = check_ptr(psi_other, "psi_other")) || (r = check_ptr(out, "out"))) return r;
    if (y && (r = check_ptr(y, "y"))) return r;
    const size_t hb = spinor_bytes(g.Vh, prec), gb = gauge_bytes(g.V, prec, link_fmt);
    if (overlap(out, hb, psi_other, hb) || overlap(out, hb, U, gb))
        return fail(LQ_ERR_ALIGN, "out overlaps psi_other or U");
    if (y && y != out && overlap(out, hb, y, hb)) return fail(LQ_ERR_ALIGN, "out partially overlaps y");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e;
    const bool dag = dagger != 0;
    if (prec == LQ_F64) e = hop_f64(g, out_parity, dag, a, b, link_fmt, U, psi_other, y, out, st);
    else if (prec == LQ_F64X) e = hop_f64x(g, out_parity, dag, a, b, link_fmt, U, psi_other, y, out, st);
    else if (prec == LQ_F32) e = hop_f32(g, out_parity, dag, a, b, link_fmt, U, psi_other, y, out, st);
    else if (prec == LQ_I32S) e = hop_i32(g, out_parity, dag, a, b, link_fmt, U, psi_other, y, out, st);
    else e = hop_f16(g, out_parity, dag, a, b, link_fmt, U, psi_other, y, out, st);
    if (e != cudaSuccess) return cuda_fail(e, "dslash_hop launch");
    return LQ_OK;
}

size_t lq_halo_face_bytes(const int32_t dims_local[4]) {
    Geom g;
    if (check_slab(dims_local, &g) != LQ_OK) return 0;
    return (size_t)g.S[3] * 96;
}

int lq_halo_pack(const int32_t dims_local[4], int32_t dagger, const void* U, const void* psi, void* to_prev,
                 void* to_next, void* cuda_stream) {
    NvtxRange nvtx("lq_halo_pack");
    Geom g;
    int r;
    if ((r = check_slab(dims_local, &g)) != LQ_OK) return r;
    if ((r = check_ptr(U, "U")) || (r = check_ptr(psi, "psi")) || (r = check_ptr(to_prev, "to_prev")) ||
        (r = check_ptr(to_next, "to_next")))
        return r;
    const size_t fb = (size_t)g.S[3] * 96, sb = spinor_bytes(g.V, LQ_F64), gb = gauge_bytes(g.V, LQ_F64, 18);
    if (overlap(to_prev, fb, to_next, fb) || overlap(to_prev, fb, psi, sb) || overlap(to_next, fb, psi, sb) ||
        overlap(to_prev, fb, U, gb) || overlap(to_next, fb, U, gb))
        return fail(LQ_ERR_ALIGN, "face buffers overlap each other or the fields");
    const cudaError_t e = halo_pack(g, dagger != 0, U, psi, to_prev, to_next, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "halo_pack launch");
    return LQ_OK;
}

int lq_halo_dslash(const int32_t dims_local[4], double m_q, int32_t dagger, const void* U, const void* psi,
                   const void* from_next, const void* from_prev, void* out, void* cuda_stream) {
    NvtxRange nvtx("lq_halo_dslash");
    Geom g;
    int r;
    if ((r = check_slab(dims_local, &g)) != LQ_OK) return r;
    if (!isfinite(m_q)) return fail(LQ_ERR_ARG, "m_q is not finite");
    if ((r = check_ptr(U, "U")) || (r = check_ptr(psi, "psi")) || (r = check_ptr(from_next, "from_next")) ||
        (r = check_ptr(from_prev, "from_prev")) || (r = check_ptr(out, "out")))
        return r;
    const size_t fb = (size_t)g.S[3] * 96, sb = spinor_bytes(g.V, LQ_F64), gb = gauge_bytes(g.V, LQ_F64, 18);
    if (overlap(out, sb, psi, sb) || overlap(out, sb, U, gb) || overlap(out, sb, from_next, fb) ||
        overlap(out, sb, from_prev, fb))
        return fail(LQ_ERR_ALIGN, "out overlaps psi, U or a face");
    const cudaError_t e =
        halo_dslash(g, m_q, dagger != 0, U, psi, from_next, from_prev, out, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "halo_dslash launch");
    return LQ_OK;
}

int lq_link_grad(const int32_t dims[4], const void* gfield, const void* psi, double scale, int32_t accumulate,
                 void* out, void* cuda_stream) {
    NvtxRange nvtx("lq_link_grad");
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (!isfinite(scale)) return fail(LQ_ERR_ARG, "scale must be finite");
    if ((r = check_ptr(gfield, "g")) || (r = check_ptr(psi, "psi")) || (r = check_ptr(out, "out"))) return r;
    const size_t sb = spinor_bytes(g.V, LQ_F64), ob = gauge_bytes(g.V, LQ_F64, LQ_LINK18);
    if (overlap(out, ob, gfield, sb) || overlap(out, ob, psi, sb)) return fail(LQ_ERR_ALIGN, "out overlaps g or psi");
    const cudaError_t e = link_grad(g, gfield, psi, scale, accumulate != 0, out, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "link_grad launch");
    return LQ_OK;
}

int lq_convert_spinor(const int32_t dims[4], int32_t src_prec, int32_t src_layout, const void* src, int32_t dst_prec,
                      int32_t dst_layout, void* dst, void* cuda_stream) {
    NvtxRange nvtx("lq_convert_spinor");
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (!valid_prec(src_prec) || !valid_prec(dst_prec)) return fail(LQ_ERR_ARG, "bad precision");
    if (!valid_layout(src_layout) || !valid_layout(dst_layout)) return fail(LQ_ERR_ARG, "bad layout");
    if ((r = check_ptr(src, "src")) || (r = check_ptr(dst, "dst"))) return r;
    if (overlap(src, spinor_bytes(g.V, src_prec), dst, spinor_bytes(g.V, dst_prec)))
        return fail(LQ_ERR_ALIGN, "dst overlaps src");
    cudaError_t e = convert_spinor(g, src_prec, src_layout, src, dst_prec, dst_layout, dst, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "convert_spinor launch");
    return LQ_OK;
}

int lq_convert_spinor_multi(const int32_t dims[4], int32_t nrhs, int32_t src_prec, int32_t src_layout,
                            const void* src, int32_t dst_prec, int32_t dst_layout, void* dst, void* cuda_stream) {
    NvtxRange nvtx("lq_convert_spinor_multi");
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (nrhs < 1 || (int64_t)nrhs * g.V > kMaxSiteFields)
        return fail(LQ_ERR_ARG, "nrhs must be >= 1 with nrhs * V <= 2^28");
    if (!valid_prec(src_prec) || !valid_prec(dst_prec)) return fail(LQ_ERR_ARG, "bad precision");
    if (!valid_layout(src_layout) || !valid_layout(dst_layout)) return fail(LQ_ERR_ARG, "bad layout");
    if ((r = check_ptr(src, "src")) || (r = check_ptr(dst, "dst"))) return r;
    const int64_t n = (int64_t)g.V * nrhs;
    if (overlap(src, spinor_bytes(n, src_prec), dst, spinor_bytes(n, dst_prec))) return fail(LQ_ERR_ALIGN, "dst overlaps src");
    cudaError_t e = convert_spinor(g, src_prec, src_layout, src, dst_prec, dst_layout, dst, (cudaStream_t)cuda_stream, nrhs);
    if (e != cudaSuccess) return cuda_fail(e, "convert_spinor launch");
    return LQ_OK;
}

int lq_convert_gauge(const int32_t dims[4], int32_t src_prec, int32_t src_layout, const void* src, int32_t dst_prec,
                     int32_t dst_fmt, int32_t dst_layout, void* dst, void* cuda_stream) {
    NvtxRange nvtx("lq_convert_gauge");
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (!valid_prec(src_prec) || !valid_prec(dst_prec)) return fail(LQ_ERR_ARG, "bad precision");
    if (!valid_layout(src_layout) || !valid_layout(dst_layout)) return fail(LQ_ERR_ARG, "bad layout");
    if (!valid_fmt(dst_fmt)) return fail(LQ_ERR_ARG, "bad link format %d", (int)dst_fmt);
    if (dst_prec == LQ_F64X && dst_fmt != LQ_LINK18) return fail(LQ_ERR_ARG, "LQ_F64X fields use 18-real links");
    if ((r = check_ptr(src, "src")) || (r = check_ptr(dst, "dst"))) return r;
    if (overlap(src, gauge_bytes(g.V, src_prec, 18), dst, gauge_bytes(g.V, dst_prec, dst_fmt)))
        return fail(LQ_ERR_ALIGN, "dst overlaps src");
    cudaError_t e = convert_gauge(g, src_prec, src_layout, src, dst_prec, dst_fmt, dst_layout, dst,
                                  (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "convert_gauge launch");
    return LQ_OK;
}

size_t lq_cg_workspace_bytes_multi(const int32_t dims[4], int32_t mode, int32_t nrhs) {
    Geom g;
    if (check_dims(dims, &g) != LQ_OK || nrhs < 1) return 0;
    if (!valid_cg_mode(mode)) return 0;
    return cg_workspace_bytes(g, mode, nrhs);
}

size_t lq_cg_workspace_bytes(const int32_t dims[4], int32_t mode) { return lq_cg_workspace_bytes_multi(dims, mode, 1); }

int lq_cg_solve_multi(const int32_t dims[4], double m_q, int32_t mode, int32_t nrhs, const void* U, const void* eta,
                      void* x, const lq_cg_params* params, void* workspace, size_t ws_bytes, lq_cg_info* info,
                      void* cuda_stream) {
    NvtxRange nvtx("lq_cg_solve_multi");
    if (info && nrhs > 0) memset(info, 0, sizeof(*info) * (size_t)nrhs);
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (nrhs < 1 || (int64_t)nrhs * g.V > kMaxSiteFields)
        return fail(LQ_ERR_ARG, "nrhs must be >= 1 with nrhs * V <= 2^28");
    if (!valid_cg_mode(mode)) return fail(LQ_ERR_ARG, "bad CG mode %d", (int)mode);
    if (!isfinite(m_q)) return fail(LQ_ERR_ARG, "m_q is not finite");
    lq_cg_params prm{1e-10, 100000, 0, 0.0, 0, 0};
    if (params) prm = *params;
    if (!(prm.tol > 0.0) || !isfinite(prm.tol)) return fail(LQ_ERR_ARG, "tol must be positive and finite");
    if (prm.max_iter < 1) return fail(LQ_ERR_ARG, "max_iter must be >= 1");
    if (prm.max_cycles < 0 || prm.chunk < 0 || prm.max_inner < 0)
        return fail(LQ_ERR_ARG, "max_cycles, chunk and max_inner must be >= 0");
    if (!(prm.delta < 1.0) || !isfinite(prm.delta)) return fail(LQ_ERR_ARG, "delta must be < 1");
    {
        const int rsel = prm.flags & (LQ_CG_RHS_BLOCK_1 | LQ_CG_RHS_BLOCK_2 | LQ_CG_RHS_BLOCK_4);
        if (rsel & (rsel - 1)) return fail(LQ_ERR_ARG, "at most one LQ_CG_RHS_BLOCK_* flag");
    }
    if ((r = check_ptr(U, "U")) || (r = check_ptr(eta, "eta")) || (r = check_ptr(x, "x"))) return r;
    if ((r = check_ptr(workspace, "workspace"))) return r == LQ_ERR_ARG ? fail(LQ_ERR_WORKSPACE, "workspace is NULL") : r;
    const size_t sb = spinor_bytes((int64_t)g.V * nrhs, LQ_F64), gb = gauge_bytes(g.V, LQ_F64, 18);
    if (overlap(x, sb, eta, sb) || overlap(x, sb, U, gb) || overlap(x, sb, workspace, ws_bytes))
        return fail(LQ_ERR_ALIGN, "x overlaps eta, U or the workspace");
    if (overlap(workspace, ws_bytes, eta, sb) || overlap(workspace, ws_bytes, U, gb))
        return fail(LQ_ERR_ALIGN, "workspace overlaps eta or U");
    r = cg_solve(g, m_q, mode, nrhs, U, eta, x, prm, workspace, ws_bytes, info, (cudaStream_t)cuda_stream);
    if (info && r < 0 && info->status == 0) info->status = r;
    return r;
}

namespace {

constexpr int kMaxLattices = 8;

// lattice batches: every mode but LQ_CG_MIXED_I32
bool valid_mode(int mode) {
    return mode == LQ_CG_F64 || mode == LQ_CG_MIXED_F32 || mode == LQ_CG_MIXED_F16 || mode == LQ_CG_F64X;
}

// lattice descriptors: counts, dims, nrhs; fills gs and nr
int check_lattices(int32_t n, const lq_lattice* lats, Geom* gs, int* nr) {
    if (n < 1 || n > kMaxLattices) return fail(LQ_ERR_ARG, "n must be 1..%d lattices", kMaxLattices);
    if (!lats) return fail(LQ_ERR_ARG, "lats is NULL");
    for (int l = 0; l < n; ++l) {
        int r;
        if ((r = check_dims(lats[l].dims, &gs[l])) != LQ_OK) return r;
        const int k = lats[l].nrhs;
        if (k != 1 && k != 2 && k != 4 && k != 8) return fail(LQ_ERR_ARG, "lattice %d: nrhs must be 1, 2, 4 or 8", l);
        if ((int64_t)k * gs[l].V > kMaxSiteFields) return fail(LQ_ERR_ARG, "lattice %d: nrhs * V exceeds 2^28", l);
        nr[l] = k;
    }
    return LQ_OK;
}

}  // namespace

size_t lq_cg_workspace_bytes_lattices(int32_t n, const lq_lattice* lats, int32_t mode) {
    Geom gs[kMaxLattices];
    int nr[kMaxLattices];
    if (!valid_mode(mode) || check_lattices(n, lats, gs, nr) != LQ_OK) return 0;
    return cg_workspace_bytes_lattices(n, gs, nr, mode);
}

int lq_cg_solve_lattices(int32_t n, const lq_lattice* lats, int32_t mode, const lq_cg_params* params,
                         void* workspace, size_t ws_bytes, lq_cg_info* info, void* cuda_stream) {
    NvtxRange nvtx("lq_cg_solve_lattices");
    Geom gs[kMaxLattices];
    int nr[kMaxLattices];
    int r;
    if ((r = check_lattices(n, lats, gs, nr)) != LQ_OK) return r;
    int total = 0;
    for (int l = 0; l < n; ++l) total += nr[l];
    if (info) memset(info, 0, sizeof(*info) * (size_t)total);
    if (!valid_mode(mode)) return fail(LQ_ERR_ARG, "bad CG mode %d", (int)mode);
    lq_cg_params prm{1e-10, 100000, 0, 0.0, 0, 0};
    if (params) prm = *params;
    if (!(prm.tol > 0.0) || !isfinite(prm.tol)) return fail(LQ_ERR_ARG, "tol must be positive and finite");
    if (prm.max_iter < 1) return fail(LQ_ERR_ARG, "max_iter must be >= 1");
    if (prm.max_cycles < 0 || prm.chunk < 0 || prm.max_inner < 0)
        return fail(LQ_ERR_ARG, "max_cycles, chunk and max_inner must be >= 0");
    if (!(prm.delta < 1.0) || !isfinite(prm.delta)) return fail(LQ_ERR_ARG, "delta must be < 1");
    if (prm.flags & (LQ_CG_PROFILE | LQ_CG_NATIVE_F64 | LQ_CG_LINK18 | LQ_CG_LINK10))
        return fail(LQ_ERR_ARG,
                    "LQ_CG_PROFILE, LQ_CG_NATIVE_F64, LQ_CG_LINK18 and LQ_CG_LINK10 do not apply to lattice batches");
    {
        const int bsel = prm.flags & (LQ_CG_BLOCK_64 | LQ_CG_BLOCK_128 | LQ_CG_BLOCK_256);
        if (bsel & (bsel - 1)) return fail(LQ_ERR_ARG, "at most one LQ_CG_BLOCK_* flag");
    }
    if ((r = check_ptr(workspace, "workspace"))) return r == LQ_ERR_ARG ? fail(LQ_ERR_WORKSPACE, "workspace is NULL") : r;
    for (int l = 0; l < n; ++l) {
        if (!isfinite(lats[l].m_q)) return fail(LQ_ERR_ARG, "lattice %d: m_q is not finite", l);
        if ((r = check_ptr(lats[l].U, "U")) || (r = check_ptr(lats[l].eta, "eta")) || (r = check_ptr(lats[l].x, "x")))
            return r;
    }
    // no solution field may overlap any input, any other solution or the workspace
    for (int l = 0; l < n; ++l) {
        const size_t xb = spinor_bytes((int64_t)gs[l].V * nr[l], LQ_F64);
        if (overlap(lats[l].x, xb, workspace, ws_bytes)) return fail(LQ_ERR_ALIGN, "lattice %d: x overlaps the workspace", l);
        for (int k = 0; k < n; ++k) {
            const size_t sb = spinor_bytes((int64_t)gs[k].V * nr[k], LQ_F64), gb = gauge_bytes(gs[k].V, LQ_F64, 18);
            if (overlap(lats[l].x, xb, lats[k].eta, sb) || overlap(lats[l].x, xb, lats[k].U, gb) ||
                (k != l && overlap(lats[l].x, xb, lats[k].x, sb)))
                return fail(LQ_ERR_ALIGN, "lattice %d: x overlaps the fields of lattice %d", l, k);
            if (overlap(workspace, ws_bytes, lats[k].eta, sb) || overlap(workspace, ws_bytes, lats[k].U, gb))
                return fail(LQ_ERR_ALIGN, "workspace overlaps the fields of lattice %d", k);
        }
    }
    return cg_solve_lattices(n, gs, lats, mode, prm, workspace, ws_bytes, info, (cudaStream_t)cuda_stream);
}

size_t lq_cg_workspace_bytes_schur(const int32_t dims[4], int32_t mode, int32_t nrhs) {
    Geom g;
    if (check_dims(dims, &g) != LQ_OK || nrhs < 1 || (int64_t)nrhs * g.V > kMaxSiteFields) return 0;
    if (!valid_cg_mode(mode) || mode == LQ_CG_F64) return 0;
    return cg_workspace_bytes_schur(g, mode, nrhs);
}

int lq_cg_solve_schur(const int32_t dims[4], double m_q, int32_t mode, int32_t nrhs, const void* U, const void* b,
                      void* x, const lq_cg_params* params, void* workspace, size_t ws_bytes, lq_cg_info* info,
                      void* cuda_stream) {
    if (info && nrhs > 0) memset(info, 0, sizeof(*info) * (size_t)nrhs);
    Geom g;
    int r;
    if ((r = check_dims(dims, &g)) != LQ_OK) return r;
    if (nrhs < 1 || (int64_t)nrhs * g.V > kMaxSiteFields)
        return fail(LQ_ERR_ARG, "nrhs must be >= 1 with nrhs * V <= 2^28");
    if (!valid_cg_mode(mode)) return fail(LQ_ERR_ARG, "bad CG mode %d", (int)mode);
    if (!isfinite(m_q)) return fail(LQ_ERR_ARG, "m_q is not finite");
    lq_cg_params prm{1e-10, 100000, 0, 0.0, 0, 0};
    if (params) prm = *params;
    if (!(prm.tol > 0.0) || !isfinite(prm.tol)) return fail(LQ_ERR_ARG, "tol must be positive and finite");
    if (prm.max_iter < 1) return fail(LQ_ERR_ARG, "max_iter must be >= 1");
    if (prm.max_cycles < 0 || prm.chunk < 0 || prm.max_inner < 0)
        return fail(LQ_ERR_ARG, "max_cycles, chunk and max_inner must be >= 0");
    if (!(prm.delta < 1.0) || !isfinite(prm.delta)) return fail(LQ_ERR_ARG, "delta must be < 1");
    if ((r = check_ptr(U, "U")) || (r = check_ptr(b, "b")) || (r = check_ptr(x, "x"))) return r;
    if ((r = check_ptr(workspace, "workspace"))) return r == LQ_ERR_ARG ? fail(LQ_ERR_WORKSPACE, "workspace is NULL") : r;
    const size_t sb = spinor_bytes((int64_t)g.V * nrhs, LQ_F64), gb = gauge_bytes(g.V, LQ_F64, 18);
    if (overlap(x, sb, b, sb) || overlap(x, sb, U, gb) || overlap(x, sb, workspace, ws_bytes))
        return fail(LQ_ERR_ALIGN, "x overlaps b, U or the workspace");
    if (overlap(workspace, ws_bytes, b, sb) || overlap(workspace, ws_bytes, U, gb))
        return fail(LQ_ERR_ALIGN, "workspace overlaps b or U");
    r = cg_solve_schur(g, m_q, mode, nrhs, U, b, x, prm, workspace, ws_bytes, info, (cudaStream_t)cuda_stream);
    if (info && r < 0 && info->status == 0) info->status = r;
    return r;
}

int lq_cg_solve(const int32_t dims[4], double m_q, int32_t mode, const void* U, const void* eta, void* x,
                const lq_cg_params* params, void* workspace, size_t ws_bytes, lq_cg_info* info,
                void* cuda_stream) {
    const int r = lq_cg_solve_multi(dims, m_q, mode, 1, U, eta, x, params, workspace, ws_bytes, info, cuda_stream);
    if (info) info->status = r;
    return r;
}

const char* lq_last_error(void) { return g_err; }


long long lq_bounds_violations(unsigned long long* first) {
#ifdef LQ_BOUNDS_CHECK
    if (first) *first = ~0ull;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    long long total = 0;
    for (OobReaderFn r : lq::oob_readers()) total += r(first);
    return total;
#else
    (void)first;
    return -1;
#endif
}

const char* lq_version(void) { return "lq 0.1 (sm_103a)"; }

int dslash_apply(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt, int32_t layout, const void* U,
                 const void* psi, void* out, void* cuda_stream) {
    return lq_dslash_apply(dims, m_q, prec, link_fmt, layout, U, psi, out, cuda_stream);
}

int dslash_adjoint(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt, int32_t layout, const void* U,
                   const void* psi, void* out, void* cuda_stream) {
    return lq_dslash_adjoint(dims, m_q, prec, link_fmt, layout, U, psi, out, cuda_stream);
}

int cg_solve(const int32_t dims[4], double m_q, int32_t mode, const void* U, const void* eta, void* x,
             const lq_cg_params* params, void* workspace, size_t ws_bytes, lq_cg_info* info, void* cuda_stream) {
    return lq_cg_solve(dims, m_q, mode, U, eta, x, params, workspace, ws_bytes, info, cuda_stream);
}

}  // extern "C"
