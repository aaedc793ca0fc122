// Helpers shared by the C-ABI entry points of the plain system (api.cu) and
// of the batched arena (arena.cu): parameter conversion and checks, host
// copies of caller arrays, and the mapping of C++ errors to orbc_status.
#pragma once
#include "ensemble.cuh"

#include <functional>
#include <new>
#include <string>

#include "../../include/orbc.h"

namespace orbc {

Params to_params(const orbc_params* p);
void check_params(const Params& P);
// Validates and copies n particles given in host memory (see orbc_set_particles).
HostInstance host_instance(const Params& prm, int n, const double* pos, const double* vel, const double* ori,
                           const double* angvel, const unsigned char* type, const unsigned* id);
// Validates and copies a bond list (see orbc_set_bonds).
void host_bonds(HostInstance& h, int nb, const int* ij, const double* r0, const double* kb);
// Device status flags to an orbc_status.
int status_code(unsigned st);
// Runs f(begin, end) over chunks of [0, n) (at least grain items each) on up
// to 16 host threads; the first exception a chunk throws is rethrown here.
void parallel_for(long long n, const std::function<void(long long, long long)>& f, long long grain = 65536);

// Runs f, turning exceptions into status codes and recording the message.
template <typename F>
int guarded_call(std::string* err, F&& f) {
    auto fail = [&](int code, const char* what) {
        if (err) *err = what;
        return code;
    };
    try {
        f();
        return ORBC_OK;
    } catch (const ArgError& e) {
        return fail(ORBC_E_ARG, e.what());
    } catch (const StateError& e) {
        return fail(ORBC_E_STATE, e.what());
    } catch (const CudaError& e) {
        return fail(e.code == cudaErrorMemoryAllocation ? ORBC_E_NOMEM : ORBC_E_CUDA, e.what());
    } catch (const std::bad_alloc&) {
        return fail(ORBC_E_NOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(ORBC_E_CUDA, e.what());
    }
}

}  // namespace orbc
