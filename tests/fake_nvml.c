/* A stand-in for the four NVML functions the library reads, for the CPU tests:
   device i has a counter that starts at 1000 * (i + 1) mJ and grows by 250 mJ
   per read; device 7 reports no counter. */
static unsigned long long reads[8];
int nvmlInit_v2(void) { return 0; }
int nvmlDeviceGetHandleByIndex_v2(unsigned i, void** h) {
  if (i >= 8) return 2;
  *h = (void*)(unsigned long)(i + 1);
  return 0;
}
int nvmlDeviceGetHandleByPciBusId_v2(const char* bus, void** h) { (void)bus; (void)h; return 6; }
int nvmlDeviceGetTotalEnergyConsumption(void* h, unsigned long long* mj) {
  unsigned long i = (unsigned long)h - 1;
  if (i == 7) return 3;
  *mj = 1000ull * (i + 1) + 250ull * reads[i]++;
  return 0;
}
