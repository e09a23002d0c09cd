/* Test helper, built by tests/test_gpu_nvtx.py: an NVTX injection library
 * (loaded by the NVTX v3 headers' initialisation through
 * NVTX_INJECTION64_PATH) that writes the message of every range pushed in a
 * domain, one per line, to the file named by $CPRA_NVTX_LOG, and the line
 * "<pop>" for every pop.  Written against the callback interface the NVTX v3
 * headers define (export table NVTX_ETID_CALLBACKS, module
 * NVTX_CB_MODULE_CORE2). */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE* g_log;
static int g_domain;

static nvtxDomainHandle_t NVTX_API record_domain_create(const char* name) {
  (void)name;
  return (nvtxDomainHandle_t)&g_domain;
}

static int NVTX_API record_push(nvtxDomainHandle_t domain, const nvtxEventAttributes_t* attr) {
  (void)domain;
  if (g_log && attr && attr->messageType == NVTX_MESSAGE_TYPE_ASCII && attr->message.ascii) {
    fprintf(g_log, "%s\n", attr->message.ascii);
    fflush(g_log);
  }
  return 0;
}

static int NVTX_API record_pop(nvtxDomainHandle_t domain) {
  (void)domain;
  if (g_log) {
    fputs("<pop>\n", g_log);
    fflush(g_log);
  }
  return 0;
}

int NVTX_API InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks* cb =
      (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = NULL;
  unsigned int last = 0;
  if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE2, &table, &last)) return 0;
  if (last < NVTX_CBID_CORE2_DomainCreateA) return 0;
  const char* path = getenv("CPRA_NVTX_LOG");
  g_log = path ? fopen(path, "a") : NULL;
  if (!g_log) return 0;
  *table[NVTX_CBID_CORE2_DomainCreateA] = (NvtxFunctionPointer)record_domain_create;
  *table[NVTX_CBID_CORE2_DomainRangePushEx] = (NvtxFunctionPointer)record_push;
  *table[NVTX_CBID_CORE2_DomainRangePop] = (NvtxFunctionPointer)record_pop;
  return 1;
}
