// flbm_tune.cu -- flbm_autotune: time candidate launch settings on a context's
// own state, keep the fastest, and remember the choice in a JSON file.
//
// Every candidate computes bitwise the same update (the two-kernel, slab
// overlap and, with two arrays, pipelined and tiled schedules run the same
// per-site arithmetic; the thread-block shape and the CUDA-graph length only change
// how the same kernels are launched), so tuning changes speed, never results.
// The in-place fused schedule, which agrees only to rounding, is not a
// candidate.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "flbm_ctx.h"

using namespace flbm;
using namespace flbm::host;

namespace {

using Settings = std::map<std::string, double>;
using Cache = std::map<std::string, Settings>;

// --- the cache file: one JSON object whose members are objects of numbers,
// {"<device and problem>": {"schedule": 1, "block_x": 128, ...}, ...}
struct Reader {
    const std::string &s;
    size_t i = 0;
    void ws()
    {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) i++;
    }
    bool ch(char c)
    {
        ws();
        if (i < s.size() && s[i] == c) {
            i++;
            return true;
        }
        return false;
    }
    bool str(std::string &out)
    {
        ws();
        if (i >= s.size() || s[i] != '"') return false;
        out.clear();
        for (i++; i < s.size() && s[i] != '"'; i++) {
            if (s[i] == '\\' && i + 1 < s.size()) i++;
            out += s[i];
        }
        if (i >= s.size()) return false;
        i++;
        return true;
    }
    bool num(double &v)
    {
        ws();
        size_t j = i;
        while (j < s.size() && std::strchr("+-.0123456789eE", s[j])) j++;
        if (j == i) return false;
        const std::string t = s.substr(i, j - i);
        char *end = nullptr;
        v = std::strtod(t.c_str(), &end);
        if (end != t.c_str() + t.size()) return false;
        i = j;
        return true;
    }
};

bool parse_cache(const std::string &text, Cache &out)
{
    Reader r{text};
    if (!r.ch('{')) return false;
    if (r.ch('}')) return true;
    do {
        std::string key;
        if (!r.str(key) || !r.ch(':') || !r.ch('{')) return false;
        Settings set;
        if (!r.ch('}')) {
            do {
                std::string name;
                double v;
                if (!r.str(name) || !r.ch(':') || !r.num(v)) return false;
                set[name] = v;
            } while (r.ch(','));
            if (!r.ch('}')) return false;
        }
        out[key] = set;
    } while (r.ch(','));
    return r.ch('}');
}

std::string quoted(const std::string &k)
{
    std::string o = "\"";
    for (char c : k) {
        if (c == '"' || c == '\\') o += '\\';
        o += c;
    }
    return o + "\"";
}

std::string format_cache(const Cache &cache)
{
    std::string o = "{\n";
    size_t n = 0;
    for (const auto &e : cache) {
        o += " " + quoted(e.first) + ": {";
        size_t m = 0;
        for (const auto &kv : e.second) {
            char num[64];
            std::snprintf(num, sizeof(num), "%.10g", kv.second);
            o += quoted(kv.first) + ": " + num + (++m < e.second.size() ? ", " : "");
        }
        o += ++n < cache.size() ? "},\n" : "}\n";
    }
    return o + "}\n";
}

bool read_file(const char *path, std::string &out)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return false;
    char buf[4096];
    size_t k;
    out.clear();
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, k);
    std::fclose(f);
    return true;
}

bool write_file(const char *path, const std::string &text)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return false;
    const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
    if (std::fclose(f) != 0 || !ok) {
        std::remove(tmp.c_str());
        return false;
    }
    return std::rename(tmp.c_str(), path) == 0;
}

const char *storage_name(int s) { return s == FLBM_STORE_F32 ? "f32" : s == FLBM_STORE_F16 ? "f16" : "bf16"; }

std::string cache_key(const flbm_ctx *c)
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        std::strcpy(prop.name, "unknown device");
        prop.multiProcessorCount = 0;
    }
    char buf[512];
    const char *lat = c->lat == FLBM_D2Q9 ? "D2Q9" : "D3Q19";
    if (is_batch(c)) {
        int nrep = 0;
        int64_t sites = 0;
        flbm_batch_size(c, &nrep, &sites);
        std::snprintf(buf, sizeof(buf), "%s|%d SMs|%s|%s|batch of %d|%lld sites", prop.name, prop.multiProcessorCount,
                      lat, storage_name(c->storage), nrep, (long long)sites);
    } else {
        std::snprintf(buf, sizeof(buf), "%s|%d SMs|%s|%s|%s|%dx%dx%d", prop.name, prop.multiProcessorCount, lat,
                      storage_name(c->storage), c->streaming == FLBM_STREAM_IN_PLACE ? "in place" : "two arrays",
                      c->nx, c->ny, c->nz);
    }
    return buf;
}

const std::pair<const char *, int> kKeys[] = {{"schedule", FLBM_OPT_SCHEDULE},
                                              {"slabs", FLBM_OPT_SLABS},
                                              {"block_x", FLBM_OPT_BLOCK_X},
                                              {"block_y", FLBM_OPT_BLOCK_Y},
                                              {"graph_steps", FLBM_OPT_GRAPH_STEPS},
                                              {"pipe_lag", FLBM_OPT_PIPE_LAG}};

// apply settings through flbm_set_option (validated like a caller's); the
// block shape goes through a narrow first shape so that x * y never exceeds
// the limit in between
flbm_status apply_settings(flbm_ctx *c, const Settings &s)
{
    flbm_status st;
    if (s.count("block_x") && s.count("block_y")) {
        if ((st = flbm_set_option(c, FLBM_OPT_BLOCK_Y, 1)) != FLBM_OK) return st;
        if ((st = flbm_set_option(c, FLBM_OPT_BLOCK_X, s.at("block_x"))) != FLBM_OK) return st;
        if ((st = flbm_set_option(c, FLBM_OPT_BLOCK_Y, s.at("block_y"))) != FLBM_OK) return st;
    }
    for (const auto &k : kKeys) {
        const std::string name = k.first;
        if (name == "block_x" || name == "block_y" || !s.count(name)) continue;
        if ((st = flbm_set_option(c, k.second, s.at(name))) != FLBM_OK) return st;
    }
    return FLBM_OK;
}

// Saved simulation state that every candidate starts from.
struct Snapshot {
    flbm_ctx *c;
    void *d_pop = nullptr;          // single box: device copy of the populations
    std::vector<unsigned char> img; // batch: checkpoint image
    int64_t step = 0;
    int parity = 0;

    flbm_status take()
    {
        if (is_batch(c)) {
            size_t bytes = 0;
            flbm_status st = flbm_checkpoint(c, nullptr, &bytes);
            if (st != FLBM_OK) return st;
            img.resize(bytes);
            return flbm_checkpoint(c, img.data(), &bytes);
        }
        flbm_status st = sync_and_check(c);
        if (st != FLBM_OK) return st;
        if (cudaMalloc(&d_pop, c->pop_bytes) != cudaSuccess) {
            d_pop = nullptr;
            cudaGetLastError();
            return fail(c, FLBM_ENOMEM, "autotune needs %zu bytes of device scratch for the state", c->pop_bytes);
        }
        FLBM_CUDA(c, cudaMemcpyAsync(d_pop, c->pop, c->pop_bytes, cudaMemcpyDeviceToDevice, c->stream), "snapshot copy");
        step = c->step;
        parity = c->parity;
        return FLBM_OK;
    }
    flbm_status put_back()
    {
        if (is_batch(c)) return flbm_restore(c, img.data(), img.size());
        FLBM_CUDA(c, cudaMemcpyAsync(c->pop, d_pop, c->pop_bytes, cudaMemcpyDeviceToDevice, c->stream), "restore copy");
        c->step = step;
        c->parity = parity;
        return sync_and_check(c);
    }
    ~Snapshot()
    {
        if (d_pop) cudaFree(d_pop);
    }
};

// device milliseconds per step of `steps` steps after `warm` untimed ones
flbm_status time_steps(flbm_ctx *c, int warm, int steps, double *ms)
{
    flbm_status st = flbm_step(c, warm);
    if (st != FLBM_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(c, FLBM_ECUDA, "cudaEventCreate failed");
    }
    cudaEventRecord(e0, c->stream);
    st = flbm_step(c, steps);
    cudaEventRecord(e1, c->stream);
    if (st == FLBM_OK) st = sync_and_check(c);
    float t = 0.0f;
    if (st == FLBM_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = fail(c, FLBM_ECUDA, "cudaEventElapsedTime failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)t / steps;
    return st;
}

std::vector<Settings> candidates(const flbm_ctx *c)
{
    std::vector<Settings> out;
    const bool tiled = c->streaming == FLBM_STREAM_TWO_ARRAYS && c->lat == FLBM_D2Q9;
    if (is_batch(c)) {
        for (int g : {0, 4, 16, 64})
            out.push_back({{"schedule", (double)FLBM_SCHEDULE_TWO_KERNELS}, {"graph_steps", (double)g}});
        if (tiled)
            for (int g : {0, 4, 16, 64})
                out.push_back({{"schedule", (double)FLBM_SCHEDULE_TILED}, {"graph_steps", (double)g}});
        return out;
    }
    const int axis = c->lat == FLBM_D2Q9 ? c->ny : c->nz;
    const int shapes[3][2] = {{128, 1}, {64, 2}, {32, 4}};
    for (const auto &b : shapes) {
        for (int gs : {0, 16})
            out.push_back({{"schedule", (double)FLBM_SCHEDULE_TWO_KERNELS}, {"graph_steps", (double)gs},
                           {"block_x", (double)b[0]}, {"block_y", (double)b[1]}});
        for (int k : {4, 8})
            if (axis >= k)
                out.push_back({{"schedule", (double)FLBM_SCHEDULE_OVERLAP}, {"graph_steps", 0.0},
                               {"slabs", (double)k}, {"block_x", (double)b[0]}, {"block_y", (double)b[1]}});
    }
    // with two arrays the fused schedule is the pipelined step (one launch a
    // step, bitwise the two-kernel update; boxes with too few slices for it
    // run the two-kernel step)
    if (c->streaming == FLBM_STREAM_TWO_ARRAYS)
        out.push_back({{"schedule", (double)FLBM_SCHEDULE_FUSED}, {"graph_steps", 0.0}, {"pipe_lag", 0.0}});
    // the tiled step of a 2D box (one launch a step; bitwise the two-kernel update)
    if (tiled)
        for (int gs : {0, 16}) out.push_back({{"schedule", (double)FLBM_SCHEDULE_TILED}, {"graph_steps", (double)gs}});
    return out;
}

} // namespace

extern "C" flbm_status flbm_autotune(flbm_ctx *c, int steps, const char *cache_path)
{
    if (!c || steps < 1 || steps > 100000) return fail(c, FLBM_EINVAL, "steps must be in [1, 100000]");
    if (!view_call_allowed(c)) return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    if (!c->initialised && !is_batch(c)) return fail(c, FLBM_ESTATE, "flbm_autotune before flbm_init");
    const std::string key = cache_key(c);
    Cache cache;
    if (cache_path) {
        std::string text;
        if (read_file(cache_path, text) && !parse_cache(text, cache))
            return fail(c, FLBM_EINVAL, "autotune cache %s is not a settings file", cache_path);
        auto it = cache.find(key);
        if (it != cache.end()) {
            Settings s = it->second;
            s.erase("ms_per_step");
            return apply_settings(c, s);
        }
    }
    Snapshot snap{c};
    flbm_status st = snap.take();
    if (st != FLBM_OK) return st;
    const bool timing = c->timing;
    c->timing = false;
    const std::vector<Settings> cand = candidates(c);
    std::vector<double> best_ms(cand.size(), 1e300);
    auto trial = [&](size_t k) -> flbm_status {
        flbm_status s = apply_settings(c, cand[k]);
        if (s != FLBM_OK) return s;
        double ms = 0.0;
        // warm up past one graph length, so that a graph is captured before the timing
        const int gs = is_batch(c) ? batch_graph_steps(c) : c->graph_steps;
        if ((s = time_steps(c, 2 + gs, steps, &ms)) != FLBM_OK) return s;
        best_ms[k] = std::min(best_ms[k], ms);
        return snap.put_back();
    };
    // every candidate once, then the three fastest again
    for (size_t k = 0; k < cand.size() && st == FLBM_OK; k++) st = trial(k);
    std::vector<size_t> order(cand.size());
    for (size_t k = 0; k < order.size(); k++) order[k] = k;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return best_ms[a] < best_ms[b]; });
    for (size_t r = 0; r < std::min<size_t>(3, order.size()) && st == FLBM_OK; r++) st = trial(order[r]);
    c->timing = timing;
    if (st != FLBM_OK) return st;
    size_t win = 0;
    for (size_t k = 1; k < cand.size(); k++)
        if (best_ms[k] < best_ms[win]) win = k;
    if ((st = apply_settings(c, cand[win])) != FLBM_OK) return st;
    if (cache_path) {
        Settings s = cand[win];
        s["ms_per_step"] = best_ms[win];
        cache[key] = s;
        if (!write_file(cache_path, format_cache(cache)))
            return fail(c, FLBM_EINVAL, "could not write the autotune cache %s", cache_path);
    }
    return FLBM_OK;
}
