// lbm_step_noalloc: one time step with no device allocation at all.
//
// The regular entry points keep their per-node moment records (the scratch
// the step's two kernels exchange) in memory that lbm_create allocates.
// Some callers cannot allocate device memory on their own: a solver that is
// embedded in a host application owning every device allocation through its
// own pool, a loop on a latency budget where cudaMalloc/cudaFree would
// synchronise the device, or a process running under a fixed memory budget.
// For them this entry point advances caller-owned populations by one step
// and takes its scratch from the file-scope array below instead.
//
// Limits and behaviour:
//  - the scratch holds the moment records of at most
//    LBM_NOALLOC_MAX_NODES nodes (16 384 nodes x 61 fields + 32 doubles =
//    7 995 648 bytes); every GPU that loads this library holds the array
//    until the process exits;
//  - every call shares the one array, so calls whose work overlaps on the
//    GPU (other streams, other host threads) race on it;
//  - the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current; make that first call
//    before any stream capture.  The address is kept for the life of the
//    process, so a cudaDeviceReset of that device ends its use here;
//  - the status word is cleared at each call; the call waits for its stream
//    to read it back.
#include <cstring>
#include <mutex>
#include <string>

#include "lbm_internal.h"

namespace {

constexpr long long kMaxNodes = LBM_NOALLOC_MAX_NODES;
constexpr int kMaxFields = 61;                        // D3Q27 with 9 species
constexpr long long kRecordDoubles = kMaxNodes * kMaxFields;

// Moment records [field][node], then 32 doubles whose first int is the
// status word.
static __device__ __align__(256) double g_noalloc_scratch[kRecordDoubles + 32];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
thread_local std::string g_noalloc_error;

// Device address of the scratch array on `device` (current at the call);
// looked up once per device.
cudaError_t scratch_on(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

lbm_status noalloc_fail(lbm_status st, const std::string& msg) {
  g_noalloc_error = msg;
  return st;
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_config* cfg, const void* pops_in,
                                       void* pops_out, double* T_guess,
                                       const char** error) {
  using namespace lbm;
  if (error) *error = nullptr;
  lbm_status st = LBM_OK;
  const std::string why = validate_config(cfg);
  if (!why.empty()) st = noalloc_fail(LBM_ERR_INVALID, why);
  else if (cfg->solid_mask || cfg->face_bc[0] || cfg->face_bc[1] || cfg->face_bc[2] ||
           cfg->face_bc[3] || cfg->face_bc[4] || cfg->face_bc[5])
    st = noalloc_fail(LBM_ERR_INVALID, "lbm_step_noalloc supports periodic boxes only");
  else if (cfg->precision == LBM_FP16_OFFSET)
    st = noalloc_fail(LBM_ERR_INVALID,
                      "FP16 offset storage needs the codec a handle keeps (use lbm_create)");
  else if (!pops_in || !pops_out || !T_guess || pops_in == pops_out)
    st = noalloc_fail(LBM_ERR_INVALID, "need distinct device buffers pops_in, pops_out and T_guess");
  else if (cfg->device < 0 || cfg->device >= kMaxDevices)
    st = noalloc_fail(LBM_ERR_RANGE, "device ordinal outside 0..63");
  else {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device >= ndev)
      st = noalloc_fail(LBM_ERR_RANGE, "device " + std::to_string(cfg->device) +
                                           " is not present (" + std::to_string(ndev) +
                                           " devices)");
  }
  if (st == LBM_OK) {
    const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
    const int D = cfg->lattice == LBM_D3Q27 ? 3 : 2;
    const int NF = record_fields(D, cfg->mech.n_species);
    if (N > kMaxNodes || NF > kMaxFields)
      st = noalloc_fail(LBM_ERR_RANGE,
                        "lbm_step_noalloc handles at most " + std::to_string(kMaxNodes) +
                            " nodes (got " + std::to_string(N) +
                            "); use lbm_create/lbm_step for larger grids");
    else {
      int prev = -1;
      cudaGetDevice(&prev);
      cudaError_t e = prev != cfg->device ? cudaSetDevice(cfg->device) : cudaSuccess;
      double* scratch = nullptr;
      if (e == cudaSuccess) e = scratch_on(cfg->device, &scratch);
      cudaStream_t stream = static_cast<cudaStream_t>(cfg->stream);
      int* status = scratch ? reinterpret_cast<int*>(scratch + kRecordDoubles) : nullptr;
      if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), stream);
      if (e == cudaSuccess) {
        DevMech mech;
        build_device_mechanism(cfg->mech, mech);
        StepArgs a;
        a.src = pops_in;
        a.dst = pops_out;
        a.rec = scratch;
        a.Tfield = T_guess;
        a.status = status;
        a.g.nx = cfg->nx;
        a.g.ny = cfg->ny;
        a.g.nz = cfg->nz;
        a.g.N = N;
        fill_units(*cfg, a.un);
        e = launch_step(D, cfg->mech.n_species, kernel_precision(*cfg), mech, a, stream);
      }
      int bits = 0;
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (prev >= 0 && prev != cfg->device) cudaSetDevice(prev);
      if (e != cudaSuccess)
        st = noalloc_fail(LBM_ERR_CUDA, std::string("lbm_step_noalloc: ") + cudaGetErrorString(e));
      else if (bits & ST_NEWTON)
        st = noalloc_fail(LBM_ERR_NEWTON, "temperature Newton did not converge");
      else if (bits & ST_NONFINITE)
        st = noalloc_fail(LBM_ERR_NONFINITE, "non-finite or non-positive density or temperature");
    }
  }
  if (st != LBM_OK && error) *error = g_noalloc_error.c_str();
  return st;
}
