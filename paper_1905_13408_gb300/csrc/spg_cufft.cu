#include <dlfcn.h>

#include <mutex>

#include "spg_cufft.h"

namespace spg {

const CufftApi &cufft_api()
{
    static CufftApi c;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        c.plan3d = reinterpret_cast<decltype(c.plan3d)>(dlsym(h, "cufftPlan3d"));
        c.plan_many = reinterpret_cast<decltype(c.plan_many)>(dlsym(h, "cufftPlanMany"));
        c.set_stream = reinterpret_cast<decltype(c.set_stream)>(dlsym(h, "cufftSetStream"));
        c.exec_r2c = reinterpret_cast<decltype(c.exec_r2c)>(dlsym(h, "cufftExecR2C"));
        c.exec_c2r = reinterpret_cast<decltype(c.exec_c2r)>(dlsym(h, "cufftExecC2R"));
        c.exec_c2c = reinterpret_cast<decltype(c.exec_c2c)>(dlsym(h, "cufftExecC2C"));
        c.destroy = reinterpret_cast<decltype(c.destroy)>(dlsym(h, "cufftDestroy"));
        c.ok = c.plan3d && c.plan_many && c.set_stream && c.exec_r2c && c.exec_c2r && c.exec_c2c && c.destroy;
    });
    return c;
}

}  // namespace spg
