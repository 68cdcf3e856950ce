// Energy counter of a GPU through NVML, read-only (the paper reports the
// energy of the aggregation kernel and of the end-to-end run per device,
// Sec. 6). NVML is loaded at run time (dlopen), so the library neither links
// against it nor needs its headers; only query functions are called, no
// setting of any GPU is read-modify-written. The counter is NVML's total
// energy of the device since the driver was loaded, in millijoules; the
// energy of a piece of work is the difference of two reads around it.
#include <dlfcn.h>

#include <cstdlib>
#include <mutex>

#include "common.cuh"

namespace agg {
namespace {

// The few NVML entry points used, by their published names and signatures
// (return 0 = success; the device handle is opaque).
using nvml_ret = int;
using nvml_dev = void*;
using fn_init = nvml_ret (*)(void);
using fn_by_bus = nvml_ret (*)(const char*, nvml_dev*);
using fn_by_index = nvml_ret (*)(unsigned, nvml_dev*);
using fn_energy = nvml_ret (*)(nvml_dev, unsigned long long*);

struct Nvml {
  bool tried = false, ok = false;
  fn_by_bus by_bus = nullptr;
  fn_by_index by_index = nullptr;
  fn_energy energy = nullptr;
  std::string why;
};

std::mutex g_nvml_mu;
Nvml g_nvml;

// Load NVML once: AGG_NVML_LIB names another library to load (a test stand-in).
Nvml& nvml() {
  Nvml& n = g_nvml;
  if (n.tried) return n;
  n.tried = true;
  const char* path = std::getenv("AGG_NVML_LIB");
  void* h = dlopen(path && *path ? path : "libnvidia-ml.so.1", RTLD_NOW | RTLD_LOCAL);
  if (!h) {
    n.why = std::string("cannot load NVML: ") + dlerror();
    return n;
  }
  fn_init init = (fn_init)dlsym(h, "nvmlInit_v2");
  n.by_bus = (fn_by_bus)dlsym(h, "nvmlDeviceGetHandleByPciBusId_v2");
  n.by_index = (fn_by_index)dlsym(h, "nvmlDeviceGetHandleByIndex_v2");
  n.energy = (fn_energy)dlsym(h, "nvmlDeviceGetTotalEnergyConsumption");
  if (!init || !n.by_index || !n.energy) {
    n.why = "NVML lacks nvmlInit_v2, nvmlDeviceGetHandleByIndex_v2 or nvmlDeviceGetTotalEnergyConsumption";
    return n;
  }
  const nvml_ret r = init();
  if (r != 0) {
    n.why = "nvmlInit_v2 failed with NVML status " + std::to_string(r);
    return n;
  }
  n.ok = true;
  return n;
}

}  // namespace
}  // namespace agg

extern "C" agg_status agg_energy_counter(int device, uint64_t* millijoules) {
  using namespace agg;
  clear_error();
  AGG_CHECK_ARG(millijoules != nullptr, "null output pointer");
  AGG_CHECK_ARG(device >= 0, "invalid device %d", device);
  std::lock_guard<std::mutex> lk(g_nvml_mu);
  Nvml& n = nvml();
  if (!n.ok) {
    set_error("%s", n.why.c_str());
    return AGG_ERR_CUDA;
  }
  // NVML numbers devices its own way: find the CUDA device by its PCI bus id,
  // and fall back to the same index when CUDA cannot say (no CUDA device)
  nvml_dev h = nullptr;
  char bus[64] = {0};
  nvml_ret r = -1;
  if (n.by_bus && cudaDeviceGetPCIBusId(bus, sizeof(bus), device) == cudaSuccess) r = n.by_bus(bus, &h);
  else cudaGetLastError();  // clear the error the failed query recorded
  if (r != 0) r = n.by_index((unsigned)device, &h);
  if (r != 0) {
    set_error("NVML has no handle for device %d (status %d)", device, r);
    return AGG_ERR_CUDA;
  }
  unsigned long long mj = 0;
  r = n.energy(h, &mj);
  if (r != 0) {
    set_error("nvmlDeviceGetTotalEnergyConsumption failed with NVML status %d", r);
    return AGG_ERR_CUDA;
  }
  *millijoules = (uint64_t)mj;
  return AGG_OK;
}
