/* Test helper: a minimal NVTX injection library.  NVTX loads it from
 * NVTX_INJECTION64_PATH at the first NVTX call of the process; it takes over
 * nvtxRangePushA and nvtxRangePop and writes one line per call ("push <name>"
 * or "pop") to the file named by SB_NVTX_LOG, so a test can check which ranges
 * the library opened and in what order. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE* g_log;

static int record_push(const char* name) {
  if (g_log) {
    fprintf(g_log, "push %s\n", name);
    fflush(g_log);
  }
  return 0;
}

static int record_pop(void) {
  if (g_log) {
    fputs("pop\n", g_log);
    fflush(g_log);
  }
  return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable core = 0;
  unsigned int n = 0;
  if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &core, &n) || n <= NVTX_CBID_CORE_RangePop)
    return 0;
  *core[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
  *core[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
  /* every NVTX client of the process (each library built with the NVTX
     headers) initialises on its own and calls this again */
  const char* path = getenv("SB_NVTX_LOG");
  if (!g_log && path) g_log = fopen(path, "a");
  return 1;
}
