// C ABI of the MLPF forward: weight-blob parsing and upload, workspace
// management, argument validation, dispatch to the FP32 / tensor-core paths,
// the CUDA-graph cache and the host-buffer entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <tuple>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace mlpf {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

void prof_begin(Model& m, cudaStream_t st, const char* name) {
    Profile* p = m.cur_prof;
    if (!m.profile || !p) return;
    if ((int)p->ev.size() < 2 * (p->n + 1)) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        p->ev.push_back(a);
        p->ev.push_back(b);
    }
    if ((int)p->names.size() <= p->n) p->names.resize(p->n + 1);
    p->names[p->n] = name;
    cudaEventRecordWithFlags(p->ev[2 * p->n], st, cudaEventRecordExternal);
}

void prof_end(Model& m, cudaStream_t st) {
    Profile* p = m.cur_prof;
    if (!m.profile || !p) return;
    cudaEventRecordWithFlags(p->ev[2 * p->n + 1], st, cudaEventRecordExternal);
    ++p->n;
}

static void prof_destroy(Profile& p) {
    for (cudaEvent_t e : p.ev) cudaEventDestroy(e);
    p.ev.clear();
    p.names.clear();
    p.n = 0;
}

bool GraphKey::operator<(const GraphKey& o) const {
    return std::tie(prec, x, cu, lo, rg, cl, su, n_events, total, max_n, ws) <
           std::tie(o.prec, o.x, o.cu, o.lo, o.rg, o.cl, o.su, o.n_events, o.total, o.max_n, o.ws);
}

// ------------------------------------------------------------ blob parsing
static const char* REG_HEAD_NAMES[4] = {"pt", "eta", "phi", "e"};
static const int REG_HEAD_WIDTH[4] = {1, 1, 2, 1};

static std::vector<std::pair<std::string, std::vector<int>>> expected_tensors(const mlpf_config& c) {
    std::vector<std::pair<std::string, std::vector<int>>> v;
    const int d = c.d, f = c.ffn;
    auto mlp = [&](const std::string& p, int n_in, int n_out) {
        v.push_back({p + ".w1", {d, n_in}});
        v.push_back({p + ".b1", {d}});
        v.push_back({p + ".w2", {n_out, d}});
        v.push_back({p + ".b2", {n_out}});
    };
    if (c.arch == 1) {
        mlp("emb.trk", c.in_dim, d);
        mlp("emb.clu", c.in_dim, d);
    } else {
        mlp("emb", c.in_dim, d);
    }
    auto stack = [&](const std::string& p0, int n) {
        for (int l = 0; l < n; ++l) {
            const std::string p = p0 + "." + std::to_string(l) + ".";
            v.push_back({p + "ln1.g", {d}});
            v.push_back({p + "ln1.b", {d}});
            for (const char* q : {"q", "k", "v", "o"}) {
                v.push_back({p + "w" + q, {d, d}});
                v.push_back({p + "b" + q, {d}});
            }
            v.push_back({p + "ln2.g", {d}});
            v.push_back({p + "ln2.b", {d}});
            v.push_back({p + "ffn.w1", {f, d}});
            v.push_back({p + "ffn.b1", {f}});
            v.push_back({p + "ffn.w2", {d, f}});
            v.push_back({p + "ffn.b2", {d}});
        }
        v.push_back({p0 + ".lnf.g", {d}});
        v.push_back({p0 + ".lnf.b", {d}});
    };
    stack("pid", c.l_pid);
    if (c.arch != 1) mlp("remb", c.in_dim + d, d);
    stack("reg", c.l_reg);
    if (c.arch == 1) {
        mlp("head.bin", d, 1);
        mlp("head.pid", d, c.n_cls - 1);
    } else {
        mlp("head.cls", d, c.n_cls);
    }
    for (int h = 0; h < 4; ++h) mlp(std::string("head.") + REG_HEAD_NAMES[h], d, REG_HEAD_WIDTH[h]);
    return v;
}

static mlpf_status parse_blob(const uint8_t* p, size_t nbytes, Model& m) {
    size_t off = 0;
    auto need = [&](size_t k) { return off + k <= nbytes; };
    if (!need(8 + 40)) { set_error("blob truncated: header"); return MLPF_E_FORMAT; }
    if (std::memcmp(p, "MLPF", 4) != 0) { set_error("blob magic is not MLPF"); return MLPF_E_FORMAT; }
    int32_t version;
    std::memcpy(&version, p + 4, 4);
    if (version != 1 && version != 2) { set_error("unsupported blob version " + std::to_string(version)); return MLPF_E_FORMAT; }
    // version 1: 10 header words (arch 0); version 2: an arch word before n_tensors
    const int nh = version == 1 ? 10 : 11;
    if (!need(8 + 4 * (size_t)nh)) { set_error("blob truncated: header"); return MLPF_E_FORMAT; }
    int32_t h[11];
    std::memcpy(h, p + 8, 4 * (size_t)nh);
    off = 8 + 4 * (size_t)nh;
    mlpf_config c{h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7], h[8], version == 1 ? 0 : h[9]};
    const int n_tensors = h[nh - 1];
    if (c.arch != 0 && c.arch != 1) { set_error("unknown architecture in blob header"); return MLPF_E_FORMAT; }
    if (c.in_dim != 42 || c.n_cls != 6 || c.n_reg != 5 || c.d <= 0 || c.d > 256 || c.heads <= 0 ||
        c.d % c.heads != 0 || (c.d / c.heads != 16 && c.d / c.heads != 32 && c.d / c.heads != 64) ||
        c.ffn <= 0 || c.ffn > 4096 || c.l_pid < 1 || c.l_reg < 1 || c.l_pid > 16 ||
        c.l_reg > 16 || (c.act != 0 && c.act != 1)) {
        set_error("unsupported model configuration in blob header");
        return MLPF_E_FORMAT;
    }
    m.cfg = c;
    auto exp = expected_tensors(c);
    if (n_tensors != (int)exp.size()) {
        set_error("blob has " + std::to_string(n_tensors) + " tensors, expected " +
                  std::to_string(exp.size()));
        return MLPF_E_FORMAT;
    }
    for (int t = 0; t < n_tensors; ++t) {
        if (!need(48 + 12)) { set_error("blob truncated: tensor record"); return MLPF_E_FORMAT; }
        char name[49];
        std::memcpy(name, p + off, 48);
        name[48] = 0;
        off += 48;
        int32_t nd, s0, s1;
        std::memcpy(&nd, p + off, 4);
        std::memcpy(&s0, p + off + 4, 4);
        std::memcpy(&s1, p + off + 8, 4);
        off += 12;
        const auto& e = exp[t];
        if (e.first != name) { set_error(std::string("unexpected tensor ") + name + ", expected " + e.first); return MLPF_E_FORMAT; }
        if (nd != (int)e.second.size() || s0 != e.second[0] || (nd == 2 ? s1 != e.second[1] : s1 != 1)) {
            set_error(std::string("bad shape for tensor ") + name);
            return MLPF_E_FORMAT;
        }
        const size_t cnt = (size_t)s0 * (nd == 2 ? s1 : 1);
        if (!need(cnt * 4)) { set_error(std::string("blob truncated: data of ") + name); return MLPF_E_FORMAT; }
        HostTensor ht;
        ht.shape = e.second;
        ht.data.resize(cnt);
        std::memcpy(ht.data.data(), p + off, cnt * 4);
        off += cnt * 4;
        m.host[name] = std::move(ht);
    }
    if (off != nbytes) { set_error("trailing bytes after the last tensor"); return MLPF_E_FORMAT; }
    return MLPF_OK;
}

mlpf_status parse_blob_into(const uint8_t* p, size_t nbytes, Model& m) { return parse_blob(p, nbytes, m); }

static mlpf_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MLPF_E_OOM : MLPF_E_CUDA;
}

#define CK(call)                                           \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return cuda_fail(_e, #call); \
    } while (0)

static mlpf_status upload_f32(Model& m) {
    const mlpf_config& c = m.cfg;
    size_t count = 0;
    for (auto& kv : m.host) count += (kv.second.data.size() + 63) / 64 * 64;
    const int d = c.d;
    count += (size_t)(c.l_pid + c.l_reg) * ((3 * d * d + 63) / 64 * 64 + (3 * d + 63) / 64 * 64);
    CK(cudaMalloc(&m.w.f32_base, count * sizeof(float)));
    std::vector<float> img(count, 0.f);
    size_t off = 0;
    for (auto& kv : m.host) {
        std::copy(kv.second.data.begin(), kv.second.data.end(), img.begin() + off);
        m.w.f32[kv.first] = m.w.f32_base + off;
        off += (kv.second.data.size() + 63) / 64 * 64;
    }
    auto cat = [&](const std::string& p, std::vector<float*>& wv, std::vector<float*>& bv) {
        size_t wo = off;
        for (const char* q : {"wq", "wk", "wv"}) {
            auto& t = m.host.at(p + q).data;
            std::copy(t.begin(), t.end(), img.begin() + off);
            off += t.size();
        }
        off = wo + (3 * d * d + 63) / 64 * 64;
        size_t bo = off;
        for (const char* q : {"bq", "bk", "bv"}) {
            auto& t = m.host.at(p + q).data;
            std::copy(t.begin(), t.end(), img.begin() + off);
            off += t.size();
        }
        off = bo + (3 * d + 63) / 64 * 64;
        wv.push_back(m.w.f32_base + wo);
        bv.push_back(m.w.f32_base + bo);
    };
    for (int l = 0; l < c.l_pid; ++l) cat("pid." + std::to_string(l) + ".", m.w.wqkv_pid, m.w.bqkv_pid);
    for (int l = 0; l < c.l_reg; ++l) cat("reg." + std::to_string(l) + ".", m.w.wqkv_reg, m.w.bqkv_reg);
    CK(cudaMemcpy(m.w.f32_base, img.data(), count * sizeof(float), cudaMemcpyHostToDevice));
    return MLPF_OK;
}

// ---------------------------------------------------------------- workspace
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static mlpf_status ensure_workspace(Model& m, int total, int n_events, bool tc) {
    Workspace& w = m.ws;
    const bool fits = (size_t)total <= w.cap_total && (size_t)n_events <= w.cap_events &&
                      (!tc || (m.tc_supported ? w.tz != nullptr : w.a16 != nullptr)) && w.base != nullptr;
    if (fits) return MLPF_OK;
    // grow geometrically; keep both paths' buffers in one allocation
    const size_t cap_t = std::max<size_t>({(size_t)total, w.cap_total * 5 / 4, 1024});
    const size_t cap_e = std::max<size_t>({(size_t)n_events, w.cap_events * 5 / 4, 16});
    const bool want_tc = (tc && m.tc_supported) || w.tz != nullptr;
    const bool want_wide = (tc && !m.tc_supported) || w.a16 != nullptr;
    if (w.base) {
        cudaFree(w.base);
        w = Workspace{};
    }
    for (auto& g : m.graphs) { cudaGraphExecDestroy(g.second.exec); prof_destroy(g.second.prof); }
    m.graphs.clear();
    m.last_prof = nullptr;
    const mlpf_config& c = m.cfg;
    const size_t d = c.d, F = c.ffn;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 1024); return o; };
    const size_t o_z = take(cap_t * d * 4), o_zn = take(cap_t * d * 4), o_qkv = take(cap_t * 3 * d * 4),
                 o_o = take(cap_t * d * 4), o_hid = take(cap_t * std::max(F, d) * 4),
                 o_hp = take(cap_t * d * 4), o_hr = take(cap_t * d * 4), o_raw = take(cap_t * 5 * 4);
    const int64_t tpad = (int64_t)align_up(cap_t + 64 * cap_e, 128);
    size_t o_tz = 0, o_tq = 0, o_tk = 0, o_to = 0, o_tvt = 0, o_thp = 0, o_blk = 0, o_kmax = 0, o_items = 0;
    if (want_tc) {
        o_tz = take(tpad * 64 * 4);
        o_tq = take(tpad * 64 * 2);
        o_tk = take(tpad * 64 * 2);
        o_to = take(tpad * 64 * 2);
        o_tvt = take(tpad * 64 * 2);
        o_thp = take(tpad * 64 * 2);
        o_blk = take((tpad / 64) * sizeof(int4));
        o_kmax = take((tpad / 64) * 4 * sizeof(float));
        o_items = take((tpad / 128 + cap_e + 1) * sizeof(int4));
    }
    // wide path: GEMM operand scratch of the widest linear-layer input (42 + d, d or FFN)
    const size_t a16_cols = align_up(std::max<size_t>({42 + d, d, F}), 64);
    const size_t o_a16 = want_wide ? take(cap_t * a16_cols * 2) : 0;
    const size_t o_b16 = want_wide ? take(cap_t * a16_cols * 2) : 0;
    const size_t o_qkv16 = want_wide ? take(cap_t * 3 * d * 2) : 0;
    const size_t o_cnt = take(64 * sizeof(int));
    const size_t o_hx = take(cap_t * 42 * 4), o_hcu = take((cap_e + 1) * 4), o_hcc = take((cap_e + 17) * 4),
                 o_hlo = take(cap_t * 6 * 4), o_hrg = take(cap_t * 5 * 4), o_hcl = take(cap_t * 4),
                 o_hsu = take(cap_e * 3 * 8);
    const size_t o_perm = take(cap_t * 4), o_xs = take(cap_t * 42 * 4), o_los = take(cap_t * 6 * 4),
                 o_rgs = take(cap_t * 5 * 4);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    char* b = (char*)base;
    w.base = base;
    w.bytes = off;
    w.cap_total = cap_t;
    w.cap_events = cap_e;
    w.z = (float*)(b + o_z); w.zn = (float*)(b + o_zn); w.qkv = (float*)(b + o_qkv);
    w.o = (float*)(b + o_o); w.hid = (float*)(b + o_hid); w.hpid = (float*)(b + o_hp);
    w.hreg = (float*)(b + o_hr); w.raw = (float*)(b + o_raw);
    w.counters = (int*)(b + o_cnt);
    if (want_wide) {
        w.a16 = (uint16_t*)(b + o_a16);
        w.b16 = (uint16_t*)(b + o_b16);
        w.qkv16 = (uint16_t*)(b + o_qkv16);
    }
    w.hx = (float*)(b + o_hx); w.hcu = (int32_t*)(b + o_hcu); w.hlogits = (float*)(b + o_hlo);
    w.hcu_chunks = (int32_t*)(b + o_hcc);
    w.hreg_out = (float*)(b + o_hrg); w.hcls = (int32_t*)(b + o_hcl); w.hsums = (double*)(b + o_hsu);
    w.perm = (int32_t*)(b + o_perm); w.xs = (float*)(b + o_xs); w.los = (float*)(b + o_los);
    w.rgs = (float*)(b + o_rgs);
    if (want_tc) {
        w.cap_tpad = tpad;
        w.tz = (float*)(b + o_tz);
        w.tq = (__nv_bfloat16*)(b + o_tq);
        w.tk = (__nv_bfloat16*)(b + o_tk);
        w.to = (__nv_bfloat16*)(b + o_to);
        w.tvt = (__nv_bfloat16*)(b + o_tvt);
        w.thp = (__nv_bfloat16*)(b + o_thp);
        w.blk = (int4*)(b + o_blk);
        w.kmax = (float*)(b + o_kmax);
        w.items = (int4*)(b + o_items);
        CK(cudaMemset(w.tvt, 0, tpad * 64 * 2));
        if (!tc_make_maps(m)) return MLPF_E_CUDA;
    }
    CK(cudaMemset(w.counters, 0, 64 * sizeof(int)));
    return MLPF_OK;
}

static mlpf_status validate(const Model* m, int32_t prec, const void* x, const void* cu,
                            int32_t n_events, int32_t total, int32_t max_n, const void* logits,
                            const void* reg) {
    if (!m) { set_error("model is NULL"); return MLPF_E_INVALID; }
    if (prec < 0 || prec > 3) { set_error("unknown precision " + std::to_string(prec)); return MLPF_E_INVALID; }
    if (n_events < 0 || total < 0 || max_n < 0) { set_error("negative size"); return MLPF_E_INVALID; }
    if (max_n > 65536) { set_error("max_n above 65536"); return MLPF_E_INVALID; }
    if (total > 0 && max_n == 0) { set_error("max_n = 0 with total > 0"); return MLPF_E_INVALID; }
    if (total > 0 && n_events == 0) { set_error("total > 0 with no events"); return MLPF_E_INVALID; }
    if (total > 0 && (!x || !cu || !logits || !reg)) { set_error("NULL input or output pointer"); return MLPF_E_INVALID; }
    if (n_events > 0 && !cu) { set_error("cu_seqlens is NULL"); return MLPF_E_INVALID; }
    if (total > 0 && ((uintptr_t)x & 7)) { set_error("x is not 8-byte aligned"); return MLPF_E_INVALID; }
    if (prec != MLPF_FP32 && !m->tc_supported && !(m->wide_supported && prec != MLPF_FP8)) {
        set_error(prec == MLPF_FP8 ? "MLPF_FP8 is built for the d=64, 4 heads, FFN 256, arch 0 model only"
                                   : "no tensor-core path for this model on this device");
        return MLPF_E_UNSUPPORTED;
    }
    if (m->attn_window > 0 && max_n > 16384) {
        set_error("windowed attention sorts events of at most 16384 elements");
        return MLPF_E_UNSUPPORTED;
    }
    if (prec == MLPF_FP8 && !m->fp8_ready) {
        set_error("MLPF_FP8 needs activation scales: call mlpf_calibrate_fp8 first");
        return MLPF_E_INVALID;
    }
    return MLPF_OK;
}

static mlpf_status launch_sequence(Model& m, int32_t prec, const float* x, const int32_t* cu,
                                   int32_t n_events, int32_t total, int32_t max_n, float* logits,
                                   float* reg, int32_t* cls, double* sums, cudaStream_t st,
                                   int64_t& launches) {
    int64_t n = 0;
    if (total > 0) {
        // windowed attention: run the forward on each event's elements in eta order
        // and scatter the outputs back to the input order
        const bool win = m.attn_window > 0;
        const float* xin = x;
        float *lo = logits, *rg = reg;
        if (win) {
            n = run_eta_order(m, x, cu, n_events, total, st);
            xin = m.ws.xs;
            lo = m.ws.los;
            rg = m.ws.rgs;
        }
        const int64_t k = n < 0 ? -1
                          : (prec == MLPF_FP32)
                                ? run_forward_f32(m, xin, cu, n_events, total, max_n, lo, rg, st)
                          : m.tc_supported ? run_forward_tc(m, prec, xin, cu, n_events, total, max_n, lo, rg, st)
                                           : run_forward_wide(m, prec, xin, cu, n_events, total, max_n, lo, rg, st);
        if (k < 0) {
            set_error(std::string("kernel launch failed: ") + cudaGetErrorString(cudaGetLastError()));
            return MLPF_E_CUDA;
        }
        n += k;
        if (win) {
            scatter_outputs(m.ws.perm, m.ws.los, m.ws.rgs, logits, reg, total, st);
            ++n;
        }
    } else if (sums && n_events > 0) {
        cudaMemsetAsync(sums, 0, (size_t)n_events * 3 * sizeof(double), st);
    }
    if (total > 0) {
        int64_t k = run_event_sums(m, cu, n_events, logits, reg, cls, sums, m.cfg.n_cls, st);
        if (k < 0) { set_error("event-sum launch failed"); return MLPF_E_CUDA; }
        n += k;
    }
    launches = n;
    return MLPF_OK;
}

static mlpf_status forward_impl(Model& m, int32_t prec, const float* x, const int32_t* cu,
                                int32_t n_events, int32_t total, int32_t max_n, float* logits,
                                float* reg, int32_t* cls, double* sums, cudaStream_t st) {
    CK(cudaSetDevice(m.device));
    mlpf_status s = ensure_workspace(m, total, n_events, prec != MLPF_FP32);
    if (s != MLPF_OK) return s;
    if (total == 0) {
        if (sums && n_events > 0) CK(cudaMemsetAsync(sums, 0, (size_t)n_events * 3 * sizeof(double), st));
        m.last_launches = 0;
        return MLPF_OK;
    }
    if (!m.use_graphs) {
        int64_t n = 0;
        m.direct_prof.n = 0;
        m.cur_prof = &m.direct_prof;
        s = launch_sequence(m, prec, x, cu, n_events, total, max_n, logits, reg, cls, sums, st, n);
        m.cur_prof = nullptr;
        m.last_prof = &m.direct_prof;
        m.last_launches = n;
        return s;
    }
    GraphKey key{prec, x, cu, logits, reg, cls, sums, n_events, total, max_n, m.ws.base};
    auto it = m.graphs.find(key);
    if (it == m.graphs.end()) {
        if (m.graphs.size() >= 16) {
            auto victim = m.graphs.begin();
            if (m.last_prof == &victim->second.prof) m.last_prof = nullptr;
            cudaGraphExecDestroy(victim->second.exec);
            prof_destroy(victim->second.prof);
            m.graphs.erase(victim);
        }
        if (!m.cap_stream) CK(cudaStreamCreateWithFlags(&m.cap_stream, cudaStreamNonBlocking));
        Profile prof;
        m.cur_prof = &prof;
        CK(cudaStreamBeginCapture(m.cap_stream, cudaStreamCaptureModeThreadLocal));
        int64_t n = 0;
        mlpf_status ls = launch_sequence(m, prec, x, cu, n_events, total, max_n, logits, reg, cls,
                                         sums, m.cap_stream, n);
        m.cur_prof = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(m.cap_stream, &g);
        if (ls != MLPF_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            prof_destroy(prof);
            return ls != MLPF_OK ? ls : cuda_fail(ce, "cudaStreamEndCapture");
        }
        cudaGraphExec_t ex = nullptr;
        ce = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { prof_destroy(prof); return cuda_fail(ce, "cudaGraphInstantiate"); }
        it = m.graphs.emplace(key, Model::GraphEntry{ex, n, prof}).first;
    }
    CK(cudaGraphLaunch(it->second.exec, st));
    m.last_launches = it->second.launches;
    m.last_prof = &it->second.prof;
    return MLPF_OK;
}

}  // namespace mlpf

using namespace mlpf;

struct mlpf_model {
    Model impl;
};

extern "C" {

mlpf_status mlpf_eval_activation(int32_t impl, int32_t act, const float* x, float* y, int32_t n, void* stream) {
    if (impl < 0 || impl > 1 || act < 0 || act > 1 || n < 0 || (n > 0 && (!x || !y))) {
        set_error("bad argument to mlpf_eval_activation");
        return MLPF_E_INVALID;
    }
    if (impl == 0) f32_eval_activation(x, y, n, act, (cudaStream_t)stream);
    else tc_eval_activation(x, y, n, act, (cudaStream_t)stream);
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_fail(e, "activation kernel");
    return MLPF_OK;
}

int32_t mlpf_abi_version(void) { return 105; }

mlpf_status mlpf_shard_events(const int32_t* sizes, int32_t n_events, int32_t n_shards, int32_t* shard_of_event,
                              double* shard_cost) {
    if (n_events < 0 || n_shards < 1 || (n_events > 0 && (!sizes || !shard_of_event))) {
        set_error("mlpf_shard_events: bad arguments");
        return MLPF_E_INVALID;
    }
    // longest processing time first: events by cost N^2 (ties: lower index first), each
    // to the shard of least cost so far (ties: lower shard index)
    std::vector<int32_t> order((size_t)n_events);
    for (int32_t e = 0; e < n_events; ++e) {
        if (sizes[e] < 0) { set_error("mlpf_shard_events: negative event size"); return MLPF_E_INVALID; }
        order[(size_t)e] = e;
    }
    auto cost = [&](int32_t e) { return (double)sizes[e] * (double)sizes[e]; };
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost(a) > cost(b); });
    std::vector<double> load((size_t)n_shards, 0.0);
    for (int32_t e : order) {
        int32_t best = 0;
        for (int32_t k = 1; k < n_shards; ++k)
            if (load[(size_t)k] < load[(size_t)best]) best = k;
        shard_of_event[e] = best;
        load[(size_t)best] += cost(e);
    }
    if (shard_cost)
        for (int32_t k = 0; k < n_shards; ++k) shard_cost[k] = load[(size_t)k];
    return MLPF_OK;
}

const char* mlpf_last_error(void) { return g_last_error.c_str(); }

mlpf_status mlpf_load_weights(const void* blob, size_t nbytes, int device, mlpf_model** out) {
    if (!blob || !out) { set_error("NULL blob or out pointer"); return MLPF_E_INVALID; }
    *out = nullptr;
    if (nbytes < 48) { set_error("blob smaller than its header"); return MLPF_E_INVALID; }
    auto* mm = new (std::nothrow) mlpf_model();
    if (!mm) { set_error("host allocation failed"); return MLPF_E_OOM; }
    Model& m = mm->impl;
    m.device = device;
    // the blob is parsed on the host first, so format errors need no GPU
    mlpf_status s = parse_blob((const uint8_t*)blob, nbytes, m);
    if (s == MLPF_OK) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
            cudaGetLastError();
            set_error("no such CUDA device " + std::to_string(device));
            delete mm;
            return MLPF_E_INVALID;
        }
    }
    if (s == MLPF_OK && cudaSetDevice(device) != cudaSuccess) { set_error("cudaSetDevice failed"); s = MLPF_E_CUDA; }
    if (s == MLPF_OK) {
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, device);
        m.sm_count = prop.multiProcessorCount;
        s = upload_f32(m);
    }
    if (s == MLPF_OK) {
        cudaError_t e = cudaMalloc(&m.status, 64);
        if (e == cudaSuccess) e = cudaMemset(m.status, 0, 64);
        if (e != cudaSuccess) s = cuda_fail(e, "status word");
    }
    if (s == MLPF_OK) {
        const mlpf_config& c = m.cfg;
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, device);
        const bool arch_ok = prop.major == 10 && prop.minor == 3;
        m.tc_supported = arch_ok && c.d == 64 && c.heads == 4 && c.ffn == 256 && c.arch == 0;
        m.wide_supported = arch_ok && !m.tc_supported;
        if (m.tc_supported && !tc_prepare_weights(m)) s = MLPF_E_CUDA;
        if (m.wide_supported && !wide_prepare_weights(m)) s = MLPF_E_CUDA;
    }
    if (s != MLPF_OK) {
        if (m.w.f32_base || m.status) mlpf_free(mm);
        else delete mm;
        return s;
    }
    *out = mm;
    return MLPF_OK;
}

void mlpf_free(mlpf_model* mm) {
    if (!mm) return;
    Model& m = mm->impl;
    cudaSetDevice(m.device);
    for (auto& g : m.graphs) { cudaGraphExecDestroy(g.second.exec); prof_destroy(g.second.prof); }
    prof_destroy(m.direct_prof);
    if (m.cap_stream) cudaStreamDestroy(m.cap_stream);
    if (m.copy_in) cudaStreamDestroy(m.copy_in);
    if (m.copy_out) cudaStreamDestroy(m.copy_out);
    if (m.compute2) cudaStreamDestroy(m.compute2);
    for (cudaEvent_t e : m.chunk_ev) cudaEventDestroy(e);
    if (m.cu_pinned) cudaFreeHost(m.cu_pinned);
    if (m.jet_base) cudaFree(m.jet_base);
    if (m.ws.base) cudaFree(m.ws.base);
    if (m.ws_alt.base) cudaFree(m.ws_alt.base);
    if (m.w.f32_base) cudaFree(m.w.f32_base);
    if (m.w.img_base) cudaFree(m.w.img_base);
    if (m.w.w16_base) cudaFree(m.w.w16_base);
    if (m.w.wide_base) cudaFree(m.w.wide_base);
    if (m.w.img8_base) cudaFree(m.w.img8_base);
    if (m.w.tc_f32_base) cudaFree(m.w.tc_f32_base);
    if (m.status) cudaFree(m.status);
    if (m.amax_dev) cudaFree(m.amax_dev);
    if (m.gate.base) cudaFree(m.gate.base);
    delete mm;
}

mlpf_status mlpf_get_config(const mlpf_model* m, mlpf_config* cfg) {
    if (!m || !cfg) { set_error("NULL argument"); return MLPF_E_INVALID; }
    *cfg = m->impl.cfg;
    return MLPF_OK;
}

mlpf_status mlpf_forward(mlpf_model* mm, int32_t precision, const float* x,
                         const int32_t* cu_seqlens, int32_t n_events, int32_t total,
                         int32_t max_n, float* logits, float* reg, int32_t* cls,
                         double* event_sums, void* stream) {
    mlpf_status s = validate(mm ? &mm->impl : nullptr, precision, x, cu_seqlens, n_events, total,
                             max_n, logits, reg);
    if (s != MLPF_OK) return s;
    return forward_impl(mm->impl, precision, x, cu_seqlens, n_events, total, max_n, logits, reg,
                        cls, event_sums, (cudaStream_t)stream);
}

mlpf_status mlpf_sync(mlpf_model* mm, void* stream) {
    if (!mm) { set_error("model is NULL"); return MLPF_E_INVALID; }
    Model& m = mm->impl;
    CK(cudaSetDevice(m.device));
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, m.status, sizeof(unsigned), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaMemsetAsync(m.status, 0, sizeof(unsigned), (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (st & (ST_TIMEOUT_ATTN | ST_TIMEOUT_GEMM)) {
        set_error("a bounded device-side wait ran out (status " + std::to_string(st) + ")");
        return MLPF_E_TIMEOUT;
    }
    if (st & ST_NONFINITE) { set_error("non-finite values in the outputs"); return MLPF_E_NONFINITE; }
    return MLPF_OK;
}

mlpf_status mlpf_forward_host(mlpf_model* mm, int32_t precision, const float* x,
                              const int32_t* cu_seqlens, int32_t n_events, int32_t total,
                              int32_t max_n, float* logits, float* reg, int32_t* cls,
                              double* event_sums, void* stream) {
    mlpf_status s = validate(mm ? &mm->impl : nullptr, precision, x, cu_seqlens, n_events, total,
                             max_n, logits, reg);
    if (s != MLPF_OK) return s;
    Model& m = mm->impl;
    CK(cudaSetDevice(m.device));
    s = ensure_workspace(m, total, n_events, precision != MLPF_FP32);
    if (s != MLPF_OK) return s;
    Workspace& w = m.ws;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = (total >= 65536 && n_events >= 2) ? std::min(m.host_chunks, (int)n_events) : 1;
    if (K == 1) {
        if (total > 0) CK(cudaMemcpyAsync(w.hx, x, (size_t)total * 42 * 4, cudaMemcpyHostToDevice, st));
        if (n_events > 0)
            CK(cudaMemcpyAsync(w.hcu, cu_seqlens, (size_t)(n_events + 1) * 4, cudaMemcpyHostToDevice, st));
        s = forward_impl(m, precision, w.hx, w.hcu, n_events, total, max_n, w.hlogits, w.hreg_out,
                         cls ? w.hcls : nullptr, event_sums ? w.hsums : nullptr, st);
        if (s != MLPF_OK) return s;
        if (total > 0) {
            CK(cudaMemcpyAsync(logits, w.hlogits, (size_t)total * 6 * 4, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(reg, w.hreg_out, (size_t)total * 5 * 4, cudaMemcpyDeviceToHost, st));
            if (cls) CK(cudaMemcpyAsync(cls, w.hcls, (size_t)total * 4, cudaMemcpyDeviceToHost, st));
        }
        if (event_sums && n_events > 0)
            CK(cudaMemcpyAsync(event_sums, w.hsums, (size_t)n_events * 3 * 8, cudaMemcpyDeviceToHost, st));
        return mlpf_sync(mm, stream);
    }
    // chunks of consecutive events (at least one event each); the first and the last
    // chunk are half the size of the others (weights 1/2, 1, ..., 1, 1/2), since their
    // input and output copies are the only ones no compute overlaps
    std::vector<int> e0(K + 1);
    e0[0] = 0;
    e0[K] = n_events;
    for (int c = 1; c < K; ++c) {
        const int64_t target = K < 3 ? (int64_t)total * c / K
                                     : (int64_t)((double)total * (2.0 * c - 1.0) / (2.0 * (K - 1)));
        int e = e0[c - 1] + 1;
        while (e < n_events - (K - c) && cu_seqlens[e] < target) ++e;
        e0[c] = e;
    }
    // per-chunk cu_seqlens rebased to 0, chunk c at offset e0[c] + c, through pinned staging
    const size_t ncu = (size_t)n_events + K;
    if (m.cu_pinned_cap < ncu) {
        if (m.cu_pinned) cudaFreeHost(m.cu_pinned);
        m.cu_pinned = nullptr;
        m.cu_pinned_cap = 0;
        CK(cudaMallocHost(&m.cu_pinned, ncu * 4));
        m.cu_pinned_cap = ncu;
    }
    for (int c = 0; c < K; ++c)
        for (int i = 0; i <= e0[c + 1] - e0[c]; ++i)
            m.cu_pinned[e0[c] + c + i] = cu_seqlens[e0[c] + i] - cu_seqlens[e0[c]];
    if (!m.copy_in) CK(cudaStreamCreateWithFlags(&m.copy_in, cudaStreamNonBlocking));
    if (!m.copy_out) CK(cudaStreamCreateWithFlags(&m.copy_out, cudaStreamNonBlocking));
    // the host staging buffers of this call (in the main workspace)
    float* const hx = w.hx;
    int32_t* const hcc = w.hcu_chunks;
    float* const hlo = w.hlogits;
    float* const hrg = w.hreg_out;
    int32_t* const hcl = w.hcls;
    double* const hsu = w.hsums;
    // odd chunks on a second compute stream with a workspace of their own, sized for the
    // largest chunk before anything is launched (a workspace that grows drops the graphs)
    const bool two = m.host_streams > 1;
    if (two) {
        int max_rows = 0, max_ev = 0;
        for (int c = 0; c < K; ++c) {
            max_rows = std::max(max_rows, cu_seqlens[e0[c + 1]] - cu_seqlens[e0[c]]);
            max_ev = std::max(max_ev, e0[c + 1] - e0[c]);
        }
        std::swap(m.ws, m.ws_alt);
        s = ensure_workspace(m, max_rows, max_ev, precision != MLPF_FP32);
        std::swap(m.ws, m.ws_alt);
        if (s != MLPF_OK) return s;
        if (!m.compute2) CK(cudaStreamCreateWithFlags(&m.compute2, cudaStreamNonBlocking));
    }
    while ((int)m.chunk_ev.size() < 2 + 2 * K) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        m.chunk_ev.push_back(e);
    }
    cudaEvent_t ev_start = m.chunk_ev[0], ev_out = m.chunk_ev[1];
    // the copy streams start after the caller's earlier work on st
    CK(cudaEventRecord(ev_start, st));
    CK(cudaStreamWaitEvent(m.copy_in, ev_start, 0));
    CK(cudaStreamWaitEvent(m.copy_out, ev_start, 0));
    CK(cudaMemcpyAsync(hcc, m.cu_pinned, ncu * 4, cudaMemcpyHostToDevice, st));
    if (two) {
        // the second compute stream starts after the per-chunk offsets are on the device
        CK(cudaEventRecord(ev_start, st));
        CK(cudaStreamWaitEvent(m.compute2, ev_start, 0));
    }
    for (int c = 0; c < K; ++c) {
        const size_t r0 = (size_t)cu_seqlens[e0[c]], rows = (size_t)cu_seqlens[e0[c + 1]] - r0;
        if (rows > 0)
            CK(cudaMemcpyAsync(hx + r0 * 42, x + r0 * 42, rows * 42 * 4, cudaMemcpyHostToDevice, m.copy_in));
        CK(cudaEventRecord(m.chunk_ev[2 + 2 * c], m.copy_in));
    }
    int64_t launches = 0;
    for (int c = 0; c < K; ++c) {
        const size_t r0 = (size_t)cu_seqlens[e0[c]], rows = (size_t)cu_seqlens[e0[c + 1]] - r0;
        const int ne = e0[c + 1] - e0[c];
        const bool alt = two && (c & 1);
        cudaStream_t cs = alt ? m.compute2 : st;
        CK(cudaStreamWaitEvent(cs, m.chunk_ev[2 + 2 * c], 0));
        if (alt) std::swap(m.ws, m.ws_alt);
        s = forward_impl(m, precision, hx + r0 * 42, hcc + e0[c] + c, ne, (int32_t)rows, max_n, hlo + r0 * 6,
                         hrg + r0 * 5, cls ? hcl + r0 : nullptr, event_sums ? hsu + (size_t)e0[c] * 3 : nullptr, cs);
        if (alt) std::swap(m.ws, m.ws_alt);
        if (s != MLPF_OK) return s;
        launches += m.last_launches;
        CK(cudaEventRecord(m.chunk_ev[3 + 2 * c], cs));
        CK(cudaStreamWaitEvent(m.copy_out, m.chunk_ev[3 + 2 * c], 0));
        if (rows > 0) {
            CK(cudaMemcpyAsync(logits + r0 * 6, hlo + r0 * 6, rows * 6 * 4, cudaMemcpyDeviceToHost, m.copy_out));
            CK(cudaMemcpyAsync(reg + r0 * 5, hrg + r0 * 5, rows * 5 * 4, cudaMemcpyDeviceToHost, m.copy_out));
            if (cls) CK(cudaMemcpyAsync(cls + r0, hcl + r0, rows * 4, cudaMemcpyDeviceToHost, m.copy_out));
        }
        if (event_sums && ne > 0)
            CK(cudaMemcpyAsync(event_sums + (size_t)e0[c] * 3, hsu + (size_t)e0[c] * 3, (size_t)ne * 3 * 8,
                               cudaMemcpyDeviceToHost, m.copy_out));
    }
    m.last_launches = launches;
    CK(cudaEventRecord(ev_out, m.copy_out));
    CK(cudaStreamWaitEvent(st, ev_out, 0));
    return mlpf_sync(mm, stream);
}

mlpf_status mlpf_calibrate_fp8(mlpf_model* mm, const float* x, const int32_t* cu_seqlens,
                               int32_t n_events, int32_t total, int32_t max_n, void* stream) {
    mlpf_status s = validate(mm ? &mm->impl : nullptr, MLPF_FP16, x, cu_seqlens, n_events, total, max_n,
                             x, x);
    if (s != MLPF_OK) return s;
    if (total == 0) { set_error("calibration needs at least one element"); return MLPF_E_INVALID; }
    if (!mm->impl.tc_supported) {
        set_error("MLPF_FP8 is built for the d=64, 4 heads, FFN 256, arch 0 model only");
        return MLPF_E_UNSUPPORTED;
    }
    Model& m = mm->impl;
    CK(cudaSetDevice(m.device));
    s = ensure_workspace(m, total, n_events, true);
    if (s != MLPF_OK) return s;
    if (!m.amax_dev) CK(cudaMalloc(&m.amax_dev, 64 * sizeof(unsigned)));
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(m.amax_dev, 0, 64 * sizeof(unsigned), st));
    Workspace& w = m.ws;
    m.calibrating = true;
    m.cur_prof = nullptr;
    const int64_t n = run_forward_tc(m, MLPF_FP16, x, cu_seqlens, n_events, total, max_n, w.hlogits,
                                     w.hreg_out, st);
    m.calibrating = false;
    if (n < 0) { set_error("calibration launch failed"); return MLPF_E_CUDA; }
    unsigned host[64];
    CK(cudaMemcpyAsync(host, m.amax_dev, sizeof(host), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    s = mlpf_sync(mm, stream);
    if (s != MLPF_OK) return s;
    // static per-tensor activation scale s_a = amax / 448 (the largest finite E4M3)
    for (auto& kv : m.act_slot) {
        float a;
        std::memcpy(&a, &host[kv.second], 4);
        m.act_scale[kv.second] = a > 0.f ? a / 448.f : 1.f;
    }
    m.fp8_ready = true;
    for (auto& g : m.graphs) { cudaGraphExecDestroy(g.second.exec); prof_destroy(g.second.prof); }
    m.graphs.clear();
    m.last_prof = nullptr;
    return MLPF_OK;
}

static void drop_graphs(Model& m) {
    for (auto& g : m.graphs) { cudaGraphExecDestroy(g.second.exec); prof_destroy(g.second.prof); }
    m.graphs.clear();
    m.last_prof = nullptr;
}

static int fmt_of(int32_t prec) { return prec == MLPF_FP16 ? 1 : prec == MLPF_FP8 ? 2 : 0; }

// Generic-width models: the attention kernel (warp-level MMAs, or PV on tcgen05) timed on the
// batch, the faster kept in MLPF_OPT_WIDE_ATTN_KERNEL; cached like the fused path's variants
// (key suffix "_wide", the kernel index as the variant).
static mlpf_status autotune_wide(Model& m, int32_t precision, const float* x, const int32_t* cu_seqlens,
                                 int32_t n_events, int32_t total, int32_t max_n, const char* cache_path,
                                 cudaStream_t st, const cudaDeviceProp& prop, int bucket) {
    if (precision != MLPF_BF16 && precision != MLPF_FP16) return MLPF_OK;   // FP8: refused by the forward
    const std::string key = "sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "_" +
                            std::to_string(prop.multiProcessorCount) + "_d" + std::to_string(m.cfg.d) + "_h" +
                            std::to_string(m.cfg.heads) + "_prec" + std::to_string(precision) + "_T" +
                            std::to_string(bucket) + "_wide";
    if (cache_path) {
        FILE* fp = std::fopen(cache_path, "r");
        if (fp) {
            char k[256];
            int v;
            float ms;
            bool hit = false;
            while (!hit && std::fscanf(fp, "%255s %d %f", k, &v, &ms) == 3)
                if (key == k && (v == 0 || v == 1)) hit = true;
            std::fclose(fp);
            if (hit) {
                m.wide_attn_kernel = v;
                drop_graphs(m);
                return MLPF_OK;
            }
        }
    }
    mlpf_status s = ensure_workspace(m, total, n_events, true);
    if (s != MLPF_OK) return s;
    Workspace& w = m.ws;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = 0;
    m.cur_prof = nullptr;
    for (int v = 0; v < 2; ++v) {
        m.wide_attn_kernel = v;
        float ms_sum = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            if (run_forward_wide(m, precision, x, cu_seqlens, n_events, total, max_n, w.hlogits, w.hreg_out, st) < 0) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                set_error("autotune launch failed");
                return MLPF_E_CUDA;
            }
            cudaEventRecord(e1, st);
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_sum += ms;  // the first run warms up
        }
        if (ms_sum / 2 < best_ms) { best_ms = ms_sum / 2; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m.wide_attn_kernel = best;
    drop_graphs(m);
    if (cache_path) {
        FILE* fp = std::fopen(cache_path, "a");
        if (fp) {
            std::fprintf(fp, "%s %d %.4f\n", key.c_str(), best, best_ms);
            std::fclose(fp);
        }
    }
    return MLPF_OK;
}

mlpf_status mlpf_autotune(mlpf_model* mm, int32_t precision, const float* x, const int32_t* cu_seqlens,
                          int32_t n_events, int32_t total, int32_t max_n, const char* cache_path,
                          void* stream) {
    mlpf_status s = validate(mm ? &mm->impl : nullptr, precision, x, cu_seqlens, n_events, total, max_n, x, x);
    if (s != MLPF_OK) return s;
    if (precision == MLPF_FP32) return MLPF_OK;  // one kernel per step: nothing to choose
    if (!mm->impl.tc_supported && !mm->impl.wide_supported) return MLPF_OK;
    if (total == 0) { set_error("autotuning needs at least one element"); return MLPF_E_INVALID; }
    Model& m = mm->impl;
    CK(cudaSetDevice(m.device));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, m.device));
    int bucket = 1;
    while (bucket < total) bucket <<= 1;
    if (!m.tc_supported) return autotune_wide(m, precision, x, cu_seqlens, n_events, total, max_n, cache_path,
                                              (cudaStream_t)stream, prop, bucket);
    const std::string key = "sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "_" +
                            std::to_string(prop.multiProcessorCount) + "_d" + std::to_string(m.cfg.d) + "_prec" +
                            std::to_string(precision) + "_T" + std::to_string(bucket) + "_v" + std::to_string(MLPF_ATTN_VARIANTS);
    const int f = fmt_of(precision);
    // cache: one "key variant ms" line per tuned case
    if (cache_path) {
        FILE* fp = std::fopen(cache_path, "r");
        if (fp) {
            char k[256];
            int v;
            float ms;
            bool hit = false;
            while (!hit && std::fscanf(fp, "%255s %d %f", k, &v, &ms) == 3)
                if (key == k && v >= 0 && v < MLPF_ATTN_VARIANTS) hit = true;
            std::fclose(fp);
            if (hit) {
                m.attn_variant[f] = v;
                drop_graphs(m);
                return MLPF_OK;
            }
        }
    }
    s = ensure_workspace(m, total, n_events, true);
    if (s != MLPF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace& w = m.ws;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = 0;
    m.cur_prof = nullptr;
    for (int v = 0; v < MLPF_ATTN_VARIANTS; ++v) {
        m.attn_variant[f] = v;
        float ms_sum = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            if (run_forward_tc(m, precision, x, cu_seqlens, n_events, total, max_n, w.hlogits, w.hreg_out, st) < 0) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                set_error("autotune launch failed");
                return MLPF_E_CUDA;
            }
            cudaEventRecord(e1, st);
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_sum += ms;  // the first run warms up
        }
        if (ms_sum / 2 < best_ms) { best_ms = ms_sum / 2; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s = mlpf_sync(mm, stream);
    if (s != MLPF_OK) return s;
    m.attn_variant[f] = best;
    drop_graphs(m);
    if (cache_path) {
        FILE* fp = std::fopen(cache_path, "a");
        if (fp) {
            std::fprintf(fp, "%s %d %.4f\n", key.c_str(), best, best_ms);
            std::fclose(fp);
        }
    }
    return MLPF_OK;
}

int32_t mlpf_get_fp8_scales(const mlpf_model* mm, int32_t cap, char* names, float* scales) {
    if (!mm) { set_error("model is NULL"); return -1; }
    const Model& m = mm->impl;
    if (!m.fp8_ready) return 0;
    int i = 0;
    for (auto& kv : m.act_slot) {
        if (i < cap) {
            if (names) {
                std::memset(names + 32 * i, 0, 32);
                std::strncpy(names + 32 * i, kv.first.c_str(), 31);
            }
            if (scales) scales[i] = m.act_scale[kv.second];
        }
        ++i;
    }
    return i;
}

mlpf_status mlpf_set_option(mlpf_model* mm, int32_t option, int64_t value) {
    if (!mm) { set_error("model is NULL"); return MLPF_E_INVALID; }
    Model& m = mm->impl;
    switch (option) {
        case MLPF_OPT_USE_GRAPHS: m.use_graphs = value != 0; return MLPF_OK;
        case MLPF_OPT_WAIT_LIMIT_NS:
            if (value < 1000000 || value > 60000000000LL) { set_error("wait limit out of range"); return MLPF_E_INVALID; }
            m.wait_limit_ns = value;
            break;
        case MLPF_OPT_DEBUG_STALL: m.debug_stall = value != 0; break;
        case MLPF_OPT_PROFILE: m.profile = value != 0; break;
        case MLPF_OPT_ATTN_WINDOW:
            if (value < 0 || value > 1024) { set_error("attention window must be 0..1024"); return MLPF_E_INVALID; }
            m.attn_window = (int)value;
            break;
        case MLPF_OPT_GATE_CONFIDENCE:
            if (value < 0 || value > 1) { set_error("gate confidence mode must be 0 or 1"); return MLPF_E_INVALID; }
            m.gate_confidence = (int)value;
            return MLPF_OK;   // host-side choice: no captured graph depends on it
        case MLPF_OPT_HOST_CHUNKS:
            if (value < 1 || value > 16) { set_error("host chunks must be 1..16"); return MLPF_E_INVALID; }
            m.host_chunks = (int)value;
            return MLPF_OK;   // host-side choice
        case MLPF_OPT_HOST_STREAMS:
            if (value < 1 || value > 2) { set_error("host streams must be 1 or 2"); return MLPF_E_INVALID; }
            m.host_streams = (int)value;
            return MLPF_OK;   // host-side choice
        case MLPF_OPT_WIDE_ATTN_KERNEL:
            if (value < 0 || value > 1) { set_error("wide attention kernel must be 0 or 1"); return MLPF_E_INVALID; }
            m.wide_attn_kernel = (int)value;
            break;
        case MLPF_OPT_ATTN_VARIANT_BF16:
        case MLPF_OPT_ATTN_VARIANT_FP16:
        case MLPF_OPT_ATTN_VARIANT_FP8:
            if (value < 0 || value >= MLPF_ATTN_VARIANTS) {
                set_error("attention variant must be 0.." + std::to_string(MLPF_ATTN_VARIANTS - 1));
                return MLPF_E_INVALID;
            }
            m.attn_variant[option - MLPF_OPT_ATTN_VARIANT_BF16] = (int)value;
            break;
        case MLPF_OPT_ATTN_CTAS_PER_SM:
            if (value < 1 || value > 1) { set_error("attention runs one CTA per SM in this build"); return MLPF_E_INVALID; }
            m.attn_ctas_per_sm = (int)value;
            break;
        default: set_error("unknown or read-only option " + std::to_string(option)); return MLPF_E_INVALID;
    }
    // options baked into captured graphs: drop them
    cudaSetDevice(m.device);
    for (auto& g : m.graphs) { cudaGraphExecDestroy(g.second.exec); prof_destroy(g.second.prof); }
    m.graphs.clear();
    m.last_prof = nullptr;
    return MLPF_OK;
}

mlpf_status mlpf_get_option(const mlpf_model* mm, int32_t option, int64_t* value) {
    if (!mm || !value) { set_error("NULL argument"); return MLPF_E_INVALID; }
    const Model& m = mm->impl;
    switch (option) {
        case MLPF_OPT_USE_GRAPHS: *value = m.use_graphs; return MLPF_OK;
        case MLPF_OPT_WAIT_LIMIT_NS: *value = m.wait_limit_ns; return MLPF_OK;
        case MLPF_OPT_DEBUG_STALL: *value = m.debug_stall; return MLPF_OK;
        case MLPF_OPT_ATTN_CTAS_PER_SM: *value = m.attn_ctas_per_sm; return MLPF_OK;
        case MLPF_OPT_ATTN_KV_STAGES: {
            static const int stages[MLPF_ATTN_VARIANTS] = {4, 6, 8, 4, 8, 4, 4, 8, 4, 8};
            *value = stages[m.attn_variant[0]];
            return MLPF_OK;
        }
        case MLPF_OPT_PROFILE: *value = m.profile; return MLPF_OK;
        case MLPF_OPT_ATTN_VARIANT_BF16:
        case MLPF_OPT_ATTN_VARIANT_FP16:
        case MLPF_OPT_ATTN_VARIANT_FP8: *value = m.attn_variant[option - MLPF_OPT_ATTN_VARIANT_BF16]; return MLPF_OK;
        case MLPF_OPT_ATTN_WINDOW: *value = m.attn_window; return MLPF_OK;
        case MLPF_OPT_GATE_CONFIDENCE: *value = m.gate_confidence; return MLPF_OK;
        case MLPF_OPT_HOST_CHUNKS: *value = m.host_chunks; return MLPF_OK;
        case MLPF_OPT_HOST_STREAMS: *value = m.host_streams; return MLPF_OK;
        case MLPF_OPT_WIDE_ATTN_KERNEL: *value = m.wide_attn_kernel; return MLPF_OK;
        default: set_error("unknown option " + std::to_string(option)); return MLPF_E_INVALID;
    }
}

int64_t mlpf_last_launch_count(const mlpf_model* m) { return m ? m->impl.last_launches : -1; }

int32_t mlpf_profile_get(mlpf_model* mm, int32_t cap, char* names, float* ms) {
    if (!mm) { set_error("model is NULL"); return -1; }
    Model& m = mm->impl;
    const Profile* p = m.last_prof;
    if (!p || !m.profile) return 0;
    cudaSetDevice(m.device);
    for (int i = 0; i < p->n && i < cap; ++i) {
        if (cudaEventSynchronize(p->ev[2 * i + 1]) != cudaSuccess) { set_error("event sync failed"); return -1; }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->ev[2 * i], p->ev[2 * i + 1]) != cudaSuccess) {
            set_error("cudaEventElapsedTime failed");
            return -1;
        }
        if (ms) ms[i] = t;
        if (names) {
            std::memset(names + 32 * i, 0, 32);
            std::strncpy(names + 32 * i, p->names[i].c_str(), 31);
        }
    }
    return p->n;
}

}  // extern "C"
