// cuFFT entry points resolved at run time (dlopen), so the solver library
// has no load-time dependency on cuFFT; used by the Fourier-shell correlation
// and by the Fourier-domain data term.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

namespace spg {

struct CufftApi {
    cufftResult (*plan3d)(cufftHandle *, int, int, int, cufftType) = nullptr;
    cufftResult (*plan_many)(cufftHandle *, int, int *, int *, int, int, int *, int, int, cufftType,
                             int) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*exec_r2c)(cufftHandle, cufftReal *, cufftComplex *) = nullptr;
    cufftResult (*exec_c2r)(cufftHandle, cufftComplex *, cufftReal *) = nullptr;
    cufftResult (*exec_c2c)(cufftHandle, cufftComplex *, cufftComplex *, int) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
    bool ok = false;
};

// The process-wide table (loaded on first use; ok == false if cuFFT is missing).
const CufftApi &cufft_api();

}  // namespace spg
