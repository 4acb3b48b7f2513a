/* A minimal NVTX injection library for the tracing test: it records every
 * range push (with its name) and pop of the process into the file named by
 * the environment variable KNNQ_NVTX_LOG.  Loaded by NVTX itself when
 * NVTX_INJECTION64_PATH names it (test infrastructure only). */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *g_out;

static int NVTX_API record_push(const char *message) {
    if (g_out) {
        fprintf(g_out, "push %s\n", message ? message : "");
        fflush(g_out);
    }
    return 0;
}

static int NVTX_API record_pop(void) {
    if (g_out) {
        fprintf(g_out, "pop\n");
        fflush(g_out);
    }
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_export_table) {
    const NvtxExportTableCallbacks *cb =
        (const NvtxExportTableCallbacks *)get_export_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    const char *path = getenv("KNNQ_NVTX_LOG");
    if (!cb || !path || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size))
        return 0;
    if (size <= NVTX_CBID_CORE_RangePop) return 0;
    g_out = fopen(path, "w");
    if (!g_out) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    return 1;
}
