// NVRTC compilation of generated kernels for sm_103a, an on-disk cubin cache,
// and loading through the CUDA runtime's library API.
#include <dlfcn.h>
#include <sys/stat.h>
#include <sys/time.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <vector>

#include <nvrtc.h>

#include "ls_internal.h"

namespace ls {
namespace {

const char *kArch = "--gpu-architecture=sm_103a";

uint64_t fnv1a(const std::string &s, uint64_t h = 1469598103934665603ull)
{
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

std::string cache_dir()
{
    const char *env = std::getenv("LS_KERNEL_CACHE");
    if (env && *env) return env;
    Dl_info info;
    if (dladdr((void *)&cache_dir, &info) && info.dli_fname) {
        std::string p = info.dli_fname;
        size_t k = p.find_last_of('/');
        if (k != std::string::npos) return p.substr(0, k) + "/kcache";
    }
    return "kcache";
}

bool read_file(const std::string &path, std::vector<char> &out)
{
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    f.seekg(0, std::ios::end);
    std::streamoff n = f.tellg();
    if (n <= 0) return false;
    f.seekg(0);
    out.resize((size_t)n);
    f.read(out.data(), n);
    return (bool)f;
}

void write_file_atomic(const std::string &path, const std::vector<char> &data)
{
    std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    {
        std::ofstream f(tmp, std::ios::binary);
        if (!f) return;
        f.write(data.data(), (std::streamsize)data.size());
        if (!f) return;
    }
    std::rename(tmp.c_str(), path.c_str());
}

ls_status nvrtc_compile(const std::string &src, const std::string &tag, std::vector<char> &cubin,
                        std::string &err)
{
    nvrtcProgram prog;
    std::string fname = tag + ".cu";
    if (nvrtcCreateProgram(&prog, src.c_str(), fname.c_str(), 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        err = "nvrtcCreateProgram failed";
        return LS_ERR_COMPILE;
    }
    const char *opts[] = {kArch, "--std=c++17", "-lineinfo", "--fmad=true", "-default-device",
                          "--extra-device-vectorization"};
    nvrtcResult r = nvrtcCompileProgram(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    size_t logn = 0;
    nvrtcGetProgramLogSize(prog, &logn);
    std::string log(logn, '\0');
    if (logn) nvrtcGetProgramLog(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
        err = std::string("NVRTC: ") + nvrtcGetErrorString(r) + "\n" + log.substr(0, 4000);
        nvrtcDestroyProgram(&prog);
        return LS_ERR_COMPILE;
    }
    size_t n = 0;
    if (nvrtcGetCUBINSize(prog, &n) != NVRTC_SUCCESS || n == 0) {
        err = "nvrtcGetCUBINSize failed";
        nvrtcDestroyProgram(&prog);
        return LS_ERR_COMPILE;
    }
    cubin.resize(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    return LS_OK;
}

}  // namespace

ls_status get_cubin(const std::string &source, const std::string &tag, std::vector<char> &cubin,
                    std::string &err)
{
    int maj = 0, min = 0;
    nvrtcVersion(&maj, &min);
    const uint64_t h = fnv1a(source, fnv1a(std::string(kArch) + "/" + std::to_string(maj) + "." +
                                           std::to_string(min) + "/v1"));
    char hex[32];
    std::snprintf(hex, sizeof hex, "%016llx", (unsigned long long)h);
    const std::string dir = cache_dir();
    const std::string path = dir + "/" + tag + "_" + hex + ".cubin";
    if (read_file(path, cubin)) {
        // mark the entry as used (its modification time), so a cache that has
        // collected kernels of earlier generator versions can be pruned by age
        utimes(path.c_str(), nullptr);
        return LS_OK;
    }
    ls_status st = nvrtc_compile(source, tag, cubin, err);
    if (st != LS_OK) return st;
    mkdir(dir.c_str(), 0755);
    write_file_atomic(path, cubin);
    // the source beside its binary only on request (LS_KEEP_KERNEL_SOURCE=1):
    // ls_spline_source / ls_spline_generate_source give it without the file
    const char *keep = std::getenv("LS_KEEP_KERNEL_SOURCE");
    if (keep && keep[0] == '1')
        write_file_atomic(dir + "/" + tag + "_" + hex + ".cu", std::vector<char>(source.begin(), source.end()));
    return LS_OK;
}

ls_status compile_and_load(const std::string &source, const std::string &tag, Module &m, std::string &err)
{
    std::vector<char> cubin;
    ls_status st = get_cubin(source, tag, cubin, err);
    if (st != LS_OK) return st;
    cudaError_t ce = cudaLibraryLoadData(&m.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce != cudaSuccess) {
        err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(ce);
        return LS_ERR_CUDA;
    }
    return LS_OK;
}

}  // namespace ls
