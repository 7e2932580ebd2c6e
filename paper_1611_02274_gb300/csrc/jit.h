// jit.h -- run-time specialised kernels for registered mass-action networks.
#pragma once
#include <string>
#include <vector>

#include "launch.cuh"

namespace bode {

// True when NVRTC could be loaded.
bool jit_available();

// Launch the generated kernels of network r for (method, precision), building
// and caching them at first use.  Returns ODE_OK or an ODE_ERR_* code with a
// description in *err.
int jit_launch(const RhsEntry& r, int method, int prec, const BatchArgs& a, const LaunchCfg& c, std::string* err);

// Every system's rate constants of network r (temperatures T[nsys], the
// parameters' first row) as two-float pairs out[j * nsys + i], computed by the
// generated module of (method, precision) on stream s.
int jit_rates(const RhsEntry& r, int method, int prec, const double* T, int64_t nsys, void* out, cudaStream_t s,
              std::string* err);

// The largest block the generated kernels of a precision form launch with:
// 128 for the forms compiled with a register budget of several resident
// blocks (larger requested blocks run as 128), else 256.
int jit_max_block(int prec);

// Compile (and, with a device present, load) the generated kernels of r.
int jit_prepare(const RhsEntry& r, int method, int prec, std::string* err);

// The generated model source of network r (for inspection).
std::string jit_model_source(const RhsEntry& r);

// Compile and load a stand-alone generated device program on the current
// device (cached); *kernels receives the kernels of the name expressions.
int jit_program(const std::string& src, const std::vector<std::string>& names, std::vector<cudaKernel_t>* kernels,
                std::string* err);

}  // namespace bode
