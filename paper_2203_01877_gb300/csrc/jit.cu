// Run-time specialisation of the few-groups aggregate (the direct group-by
// of Section 5.4's aggregation, groupdirect.cuh).
//
// The generic kernel reads its query's shape -- the column types of the
// conditions, keys and sum factors, the factors' affine kinds, the counts --
// from its arguments and dispatches on them in every step.  For a large input
// the same kernel source is compiled at run time with NVRTC for that one
// shape: the shape's values become compile-time constants (DirAnySpec's
// members, returning them) and the dispatch folds away, as in a query
// compiler.  Each shape is compiled once per process; the cubins are also
// kept on disk (TQP_JIT_CACHE, else _jit_cache/ beside libtqp.so), keyed by a
// hash of the source, the options and the kernel headers.  NVRTC is loaded at
// first use (dlopen); without it, or when a compile fails, the generic kernel
// runs, with the same results.
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "groupdirect.cuh"
#include "host.h"

#ifndef TQP_CUDA_LIBDIR
#define TQP_CUDA_LIBDIR "/usr/local/cuda/lib64"
#endif

namespace tqp {
namespace {

struct NvrtcApi {
    bool ok = false;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

const NvrtcApi& nvrtc_api() {
    static const NvrtcApi api = [] {
        NvrtcApi a;
        void* h = nullptr;
        for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", TQP_CUDA_LIBDIR "/libnvrtc.so.13"})
            if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return a;
        a.create = reinterpret_cast<decltype(a.create)>(dlsym(h, "nvrtcCreateProgram"));
        a.compile = reinterpret_cast<decltype(a.compile)>(dlsym(h, "nvrtcCompileProgram"));
        a.log_size = reinterpret_cast<decltype(a.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        a.log = reinterpret_cast<decltype(a.log)>(dlsym(h, "nvrtcGetProgramLog"));
        a.cubin_size = reinterpret_cast<decltype(a.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        a.cubin = reinterpret_cast<decltype(a.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        a.destroy = reinterpret_cast<decltype(a.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        a.ok = a.create && a.compile && a.log_size && a.log && a.cubin_size && a.cubin && a.destroy;
        return a;
    }();
    return api;
}

// The directory of libtqp.so (the package): csrc/ holds the kernel headers.
std::string package_dir() {
    Dl_info info;
    if (!dladdr(reinterpret_cast<void*>(&nvrtc_api), &info) || !info.dli_fname) return "";
    const std::string p = info.dli_fname;
    const size_t k = p.rfind('/');
    return k == std::string::npos ? std::string(".") : p.substr(0, k);
}

bool read_file(const std::string& path, std::string* out) {
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return false;
    out->clear();
    char buf[65536];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) out->append(buf, n);
    fclose(f);
    return true;
}

uint64_t fnv1a(const std::string& s, uint64_t h) {
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ULL;
    }
    return h;
}

// The headers a specialised kernel includes (their text enters the cache key).
const char* const kJitHeaders[] = {"csrc/common.cuh", "csrc/engine.cuh", "csrc/group.cuh", "csrc/finalize.cuh",
                                   "csrc/groupdirect.cuh", "../include/tqp.h"};

struct JitEntry {
    int state = 0;              // 0 not compiled (yet), 1 loaded, 2 cannot be had
    bool disk_checked = false;  // the disk cache was looked at
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    uint64_t attr_devices = 0;  // devices whose shared-memory attribute is set
};

std::mutex g_mu;
// (never destroyed: loaded libraries stay valid until the process ends)
std::map<std::string, JitEntry>* g_cache = new std::map<std::string, JitEntry>();
std::atomic<long long> g_stats[4];  // compiled, loaded from disk, specialised launches, failed

// NVRTC: `src` to a cubin for sm_103a; false with the log in *log on failure.
bool nvrtc_compile(const std::string& src, const std::vector<std::string>& opts, std::string* cubin,
                   std::string* log) {
    const NvrtcApi& api = nvrtc_api();
    if (!api.ok) {
        *log = "NVRTC not found";
        return false;
    }
    nvrtcProgram prog = nullptr;
    if (api.create(&prog, src.c_str(), "tqp_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *log = "nvrtcCreateProgram failed";
        return false;
    }
    std::vector<const char*> o;
    for (const std::string& s : opts) o.push_back(s.c_str());
    const nvrtcResult r = api.compile(prog, static_cast<int>(o.size()), o.data());
    size_t n = 0;
    api.log_size(prog, &n);
    log->assign(n, '\0');
    if (n) api.log(prog, &(*log)[0]);
    bool ok = r == NVRTC_SUCCESS;
    if (ok) {
        api.cubin_size(prog, &n);
        cubin->assign(n, '\0');
        ok = n > 0 && api.cubin(prog, &(*cubin)[0]) == NVRTC_SUCCESS;
    }
    api.destroy(&prog);
    return ok;
}

std::string cache_dir(const std::string& pkg) {
    const char* env = getenv("TQP_JIT_CACHE");
    return env && *env ? std::string(env) : pkg + "/_jit_cache";
}

// The cubin of `src`: from the disk cache, else (when allowed) compiled and
// stored there.  TQP_OK with the cubin; TQP_ERR_CAPACITY: not on disk and
// compiling not allowed; other statuses: the shape cannot be compiled here.
tqp_status jit_cubin(const std::string& src, std::string* cubin, bool allow_compile) {
    const std::string pkg = package_dir();
    if (pkg.empty()) return fail(TQP_ERR_UNSUPPORTED, "run-time specialisation: libtqp.so's directory not found");
    const std::vector<std::string> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device",
                                           "-I" + pkg + "/csrc", "-I" + pkg + "/../include"};
    uint64_t h = fnv1a(src, 1469598103934665603ULL);
    for (const std::string& o : opts) h = fnv1a(o, h);
    for (const char* f : kJitHeaders) {
        std::string text;
        if (!read_file(pkg + "/" + f, &text))
            return fail(TQP_ERR_UNSUPPORTED, "run-time specialisation: kernel source %s/%s not found", pkg.c_str(), f);
        h = fnv1a(text, h);
    }
    const std::string dir = cache_dir(pkg);
    char name[64];
    snprintf(name, sizeof(name), "/%016llx.cubin", static_cast<unsigned long long>(h));
    const std::string path = dir + name;
    if (read_file(path, cubin) && !cubin->empty()) {
        ++g_stats[1];
        return TQP_OK;
    }
    if (!allow_compile) return TQP_ERR_CAPACITY;
    std::string log;
    if (!nvrtc_compile(src, opts, cubin, &log)) {
        ++g_stats[3];
        return fail(TQP_ERR_UNSUPPORTED, "run-time specialisation failed: %.900s", log.c_str());
    }
    ++g_stats[0];
    mkdir(dir.c_str(), 0755);  // (may exist; a failed store only costs a recompile later)
    const std::string tmp = path + "." + std::to_string(getpid()) + ".tmp";
    if (FILE* f = fopen(tmp.c_str(), "wb")) {
        const bool wrote = fwrite(cubin->data(), 1, cubin->size(), f) == cubin->size();
        fclose(f);
        if (!wrote || rename(tmp.c_str(), path.c_str()) != 0) unlink(tmp.c_str());
    }
    return TQP_OK;
}

// "static constexpr __device__ int name(int i) { return i == 0 ? v0 : ... : -1; }"
std::string spec_fn(const char* name, const std::vector<int>& v) {
    std::string s = std::string("    static constexpr __device__ int ") + name + "(int i) { return ";
    for (size_t i = 0; i < v.size(); ++i) s += "i == " + std::to_string(i) + " ? " + std::to_string(v[i]) + " : ";
    return s + "-1; }\n";
}

std::string spec_val(const char* name, int v) {
    return std::string("    static constexpr __device__ int ") + name + "() { return " + std::to_string(v) + "; }\n";
}

// The shape of D: what the specialised kernel fixes at compile time.
struct DirShape {
    std::vector<int> ct, kt, ft, fk, fs, mul;
    int ncond = 0, ngc = 0, nsum = 0;
};

DirShape shape_of(const GroupDirectArgs& D) {
    DirShape h;
    h.ncond = D.ncond;
    h.ngc = D.ngc;
    h.nsum = D.nsum;
    for (int c = 0; c < D.ncond; ++c) h.ct.push_back(D.cond[c].type);
    for (int i = 0; i < D.ngc; ++i) h.kt.push_back(D.key[i].type);
    for (int a = 0; a < D.nsum; ++a) h.mul.push_back(D.f[a][1].kind != kFacConst || D.f[a][1].b != 1 ? 1 : 0);
    for (int i = 0; i < 2 * D.nsum; ++i) {
        const DirFactor& f = D.f[i / 2][i % 2];
        const bool used = i % 2 == 0 || h.mul[i / 2];
        h.ft.push_back(f.type);
        h.fk.push_back(used ? f.kind : kFacConst);
        int same = -1;  // an earlier evaluated factor of the same column
        if (used && f.kind != kFacConst)
            for (int j = 0; j < i && same < 0; ++j) {
                const DirFactor& g = D.f[j / 2][j % 2];
                const bool gused = j % 2 == 0 || h.mul[j / 2];
                if (gused && g.kind != kFacConst && g.p == f.p && g.type == f.type) same = j;
            }
        h.fs.push_back(same);
    }
    return h;
}

// The shape as a short byte string (the in-process cache key).
std::string shape_key(const DirShape& h) {
    std::string k;
    auto put = [&k](int v) { k.push_back(static_cast<char>(v + 2)); };
    put(h.ncond);
    for (int v : h.ct) put(v);
    put(h.ngc);
    for (int v : h.kt) put(v);
    put(h.nsum);
    for (size_t i = 0; i < h.ft.size(); ++i) {
        put(h.ft[i]);
        put(h.fk[i]);
        put(h.fs[i]);
    }
    for (int v : h.mul) put(v);
    return k;
}

// The kernel source specialised to a shape (the sums-only kernel).
std::string dir_spec_source(const DirShape& h) {
    std::string s = "#include \"groupdirect.cuh\"\nstruct JitSpec {\n";
    s += spec_val("ncond", h.ncond) + spec_fn("cond_type", h.ct) + spec_val("ngc", h.ngc) + spec_fn("key_type", h.kt);
    s += spec_val("nsum", h.nsum) + spec_fn("fac_type", h.ft) + spec_fn("fac_kind", h.fk) + spec_fn("fac_same", h.fs);
    s += spec_fn("mul", h.mul) + "};\n";
    s += "extern \"C\" __global__ void __launch_bounds__(tqp::kDirThreads, tqp::kDirMinBlocks)\n"
         "tqp_group_direct_jit(const __grid_constant__ tqp::GroupDirectArgs A) {\n"
         "    extern __shared__ __align__(16) unsigned char dsm[];\n"
         "    tqp::group_direct_block<false, JitSpec>(A, dsm, blockIdx.x, gridDim.x);\n"
         "}\n";
    return s;
}

}  // namespace

const void* jit_group_direct(const tqp_ctx* ctx, const GroupDirectArgs& D, long long rows) {
    if (ctx->jit == 0) return nullptr;
    const bool may_compile = ctx->jit == 2 || rows >= kJitMinRows;
    const DirShape h = shape_of(D);
    const std::string key = shape_key(h);
    std::lock_guard<std::mutex> lk(g_mu);
    JitEntry& e = (*g_cache)[key];
    if (e.state == 0 && (may_compile || !e.disk_checked)) {
        std::string cubin;
        const tqp_status st = jit_cubin(dir_spec_source(h), &cubin, may_compile);
        e.disk_checked = true;
        if (st == TQP_OK) {
            const bool ok =
                cudaLibraryLoadData(&e.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) == cudaSuccess &&
                cudaLibraryGetKernel(&e.kernel, e.lib, "tqp_group_direct_jit") == cudaSuccess;
            e.state = ok ? 1 : 2;
            if (!ok) ++g_stats[3];
        } else if (st != TQP_ERR_CAPACITY) {
            e.state = 2;
        }
        // a shape that cannot be specialised runs the generic kernel: not the caller's error
        (void)cudaGetLastError();
        clear_error();
    }
    if (e.state != 1) return nullptr;
    const void* k = reinterpret_cast<const void*>(e.kernel);
    const uint64_t bit = ctx->device < 64 ? 1ULL << ctx->device : 0;
    if (!(e.attr_devices & bit)) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kDirSmemBytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        e.attr_devices |= bit;
    }
    return k;
}

void jit_count_launch() { ++g_stats[2]; }

}  // namespace tqp

using namespace tqp;

tqp_status tqp_ctx_set_jit(tqp_ctx* ctx, int32_t mode) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (mode < 0 || mode > 2) return fail(TQP_ERR_INVALID_ARG, "jit mode must be 0, 1 or 2");
    ctx->jit = mode;
    return TQP_OK;
}

void tqp_jit_stats(int64_t* out) {
    if (!out) return;
    for (int i = 0; i < 4; ++i) out[i] = g_stats[i].load();
}

tqp_status tqp_jit_probe(void) {
    clear_error();
    // a sample shape: one int32 condition, two uint8 keys, the sums x, y and
    // y * (100 - z) over an int32 and two int64 columns (pointers only compared)
    GroupDirectArgs D;
    memset(&D, 0, sizeof(D));
    D.ncond = 1;
    D.cond[0].type = TQP_I32;
    D.ngc = 2;
    D.key[0].type = D.key[1].type = TQP_U8;
    D.nsum = 3;
    const unsigned char* col[3] = {reinterpret_cast<const unsigned char*>(16),
                                   reinterpret_cast<const unsigned char*>(32),
                                   reinterpret_cast<const unsigned char*>(48)};
    const int type[3] = {TQP_I32, TQP_I64, TQP_I64};
    for (int a = 0; a < 3; ++a) {
        D.f[a][0] = DirFactor{col[a == 0 ? 0 : 1], type[a == 0 ? 0 : 1], kFacPlain, 1, 0, 0, 0};
        D.f[a][1] = DirFactor{nullptr, TQP_I64, kFacConst, 0, 1, 0, 0};
    }
    D.f[2][1] = DirFactor{col[2], type[2], kFacRsub, 1, 100, 0, 0};
    std::string cubin;
    return jit_cubin(dir_spec_source(shape_of(D)), &cubin, true);
}
