// Multi-lattice solves: workspace layout, mode dispatch, and the tuning cache (the inner
// block size of a lattice batch, the right-hand sides per thread of a batched solve).
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>

#include "solver_lattices.cuh"

namespace lq {

namespace solver_detail {

namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

const char* tune_path() {
    const char* p = getenv("LQ_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

bool valid_block(int b) { return b == 64 || b == 128 || b == 256; }

// a stored value is a block size, or right-hand sides per thread for the keys of
// tune_key_rhs_block
bool valid_value(const std::string& key, int v) {
    if (key.find("\"what\":\"rhs_block\"") != std::string::npos) return v == 1 || v == 2 || v == 4;
    return valid_block(v);
}

// cache file: one JSON object per line, {"block": N, "key": {...}}; N is the tuned value (a
// block size, or right-hand sides per thread for the keys of tune_key_rhs_block)
void load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = tune_path();
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[4096];
    while (fgets(line, sizeof line, f)) {
        int bs = 0, used = 0;
        if (sscanf(line, "{\"block\": %d, \"key\": %n", &bs, &used) < 1 || used == 0) continue;
        std::string key(line + used);
        while (!key.empty() && (key.back() == '\n' || key.back() == '\r' || key.back() == ' ')) key.pop_back();
        if (key.empty() || key.back() != '}') continue;
        key.pop_back();
        if (valid_value(key, bs)) g_tune[key] = bs;
    }
    fclose(f);
}

}  // namespace

bool tune_lookup(const std::string& key, int* block) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_locked();
    const auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *block = it->second;
    return true;
}

void tune_store(const std::string& key, int block) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_locked();
    g_tune[key] = block;
    if (const char* path = tune_path()) {
        if (FILE* f = fopen(path, "a")) {
            fprintf(f, "{\"block\": %d, \"key\": %s}\n", block, key.c_str());
            fclose(f);
        }
    }
}

namespace {

// {"gpu":"<name>","sm":<major minor>, -- the start of every key, for the current device
std::string tune_key_gpu() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = "unknown";
    int sm = 0;
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        name = prop.name;
        sm = prop.major * 10 + prop.minor;
    }
    for (char& c : name)
        if (c == '"' || c == '\\') c = '\'';
    return "{\"gpu\":\"" + name + "\",\"sm\":" + std::to_string(sm) + ",";
}

}  // namespace

std::string tune_key_rhs_block(int ip, int fmt, int hp, const Geom& g, int nb) {
    return tune_key_gpu() + "\"what\":\"rhs_block\",\"inner\":" + std::to_string(ip) + ",\"links\":" +
           std::to_string(fmt) + ",\"outer\":" + std::to_string(hp) + ",\"dims\":[" + std::to_string(g.L[0]) + "," +
           std::to_string(g.L[1]) + "," + std::to_string(g.L[2]) + "," + std::to_string(g.L[3]) + "],\"nrhs\":" +
           std::to_string(nb) + "}";
}

std::string tune_key(int mode, int n, const LatticeJob* jobs) {
    std::string k = tune_key_gpu() + "\"mode\":" + std::to_string(mode) + ",\"lattices\":[";
    for (int l = 0; l < n; ++l) {
        if (l) k += ",";
        k += "[" + std::to_string(jobs[l].g.L[0]) + "," + std::to_string(jobs[l].g.L[1]) + "," +
             std::to_string(jobs[l].g.L[2]) + "," + std::to_string(jobs[l].g.L[3]) + "," + std::to_string(jobs[l].nb) +
             "]";
    }
    return k + "]}";
}

// Workspace of lattice l starts at the sum of the earlier lattices' (256-byte aligned) sizes.
size_t lattice_layouts(int n, const Geom* gs, const int* nrhs, int mode, LatticeJob* jobs) {
    const bool pairs = mode != LQ_CG_F64;
    size_t off = 0;
    for (int l = 0; l < n; ++l) {
        const WsLayout w = ws_layout(gs[l], mode, pairs, 12, nrhs[l]);
        if (jobs) {
            jobs[l].w = w;
            jobs[l].off = off;
        }
        off += align256(w.total);
    }
    return off;
}

}  // namespace solver_detail

size_t cg_workspace_bytes_lattices(int n, const Geom* gs, const int* nrhs, int mode) {
    return solver_detail::lattice_layouts(n, gs, nrhs, mode, nullptr);
}

int cg_solve_lattices(int n, const Geom* gs, const lq_lattice* lats, int mode, const lq_cg_params& prm, void* ws,
                      size_t ws_bytes, lq_cg_info* info, cudaStream_t st) {
    using namespace solver_detail;
    LatticeJob jobs[kMaxLat];
    int nrhs[kMaxLat];
    for (int l = 0; l < n; ++l) nrhs[l] = lats[l].nrhs;
    const size_t need = lattice_layouts(n, gs, nrhs, mode, jobs);
    if (ws == nullptr || ws_bytes < need)
        return fail(LQ_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
    for (int l = 0; l < n; ++l) {
        jobs[l].g = gs[l];
        jobs[l].m_q = lats[l].m_q;
        jobs[l].nb = lats[l].nrhs;
        jobs[l].U = lats[l].U;
        jobs[l].eta = lats[l].eta;
        jobs[l].x = lats[l].x;
    }
    double delta = prm.delta;
    if (!(delta > 0.0)) delta = default_delta(mode);
    char* w = (char*)ws;
    switch (mode) {
        case LQ_CG_F64: return lattices_f64(n, jobs, prm, delta, w, info, st);
        case LQ_CG_F64X: return lattices_f64x(n, jobs, prm, delta, w, info, st);
        case LQ_CG_MIXED_F32: return lattices_mixed_f32(n, jobs, prm, delta, w, info, st);
        case LQ_CG_MIXED_F16: return lattices_mixed_f16(n, jobs, prm, delta, w, info, st);
        default: return fail(LQ_ERR_ARG, "unknown CG mode %d", mode);
    }
}

}  // namespace lq
