/* nvtx_count.c — test fixture: a minimal NVTX injection library.
 *
 * NVTX (header-only in the CUDA toolkit) loads the library named by the
 * environment variable NVTX_INJECTION64_PATH at the first NVTX call and calls
 * its InitializeInjectionNvtx2 with a function that returns export tables.
 * This one asks for the core module's function table and installs two
 * callbacks: RangePushA counts pushes per range name, RangePop counts pops
 * and tracks the nesting depth per thread. The tests read the counts through
 * ctypes (dlopen of the same path returns the same loaded library).
 *
 * The few type and constant definitions below restate the public NVTX v3
 * callback interface (nvtxDetail/nvtxTypes.h): the export-table id of the
 * callbacks, the core module id and the two callback ids.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

typedef void (*nc_fn)(void);
typedef nc_fn** nc_table;
typedef struct {
  size_t struct_size;
  int (*get_module_function_table)(int module, nc_table* out_table, unsigned* out_size);
} nc_callbacks;
typedef const void* (*nc_get_export_table)(uint32_t id);

enum { NC_ETID_CALLBACKS = 1, NC_MODULE_CORE = 1, NC_CBID_PUSH_A = 9, NC_CBID_POP = 11 };

#define NC_MAX_NAMES 128
#define NC_NAME_LEN 64
static char nc_names[NC_MAX_NAMES][NC_NAME_LEN];
static int nc_counts[NC_MAX_NAMES];
static int nc_n_names, nc_pops, nc_unbalanced;
static __thread int nc_depth;
static pthread_mutex_t nc_mu = PTHREAD_MUTEX_INITIALIZER;

static int nc_push_a(const char* msg) {
  pthread_mutex_lock(&nc_mu);
  int i = 0;
  while (i < nc_n_names && strncmp(nc_names[i], msg, NC_NAME_LEN - 1) != 0) ++i;
  if (i == nc_n_names && nc_n_names < NC_MAX_NAMES) {
    strncpy(nc_names[i], msg, NC_NAME_LEN - 1);
    ++nc_n_names;
  }
  if (i < NC_MAX_NAMES) ++nc_counts[i];
  pthread_mutex_unlock(&nc_mu);
  return nc_depth++;
}

static int nc_pop(void) {
  pthread_mutex_lock(&nc_mu);
  ++nc_pops;
  if (nc_depth == 0) ++nc_unbalanced;
  pthread_mutex_unlock(&nc_mu);
  if (nc_depth > 0) --nc_depth;
  return nc_depth;
}

int InitializeInjectionNvtx2(nc_get_export_table get) {
  const nc_callbacks* cb = (const nc_callbacks*)get(NC_ETID_CALLBACKS);
  nc_table table = NULL;
  unsigned size = 0;
  if (!cb || !cb->get_module_function_table(NC_MODULE_CORE, &table, &size)) return 0;
  if (size < NC_CBID_POP) return 0;
  *table[NC_CBID_PUSH_A] = (nc_fn)nc_push_a;
  *table[NC_CBID_POP] = (nc_fn)nc_pop;
  return 1;
}

/* Read by the tests. */
int nvtx_count_of(const char* name) {
  pthread_mutex_lock(&nc_mu);
  int n = 0;
  for (int i = 0; i < nc_n_names; ++i)
    if (strncmp(nc_names[i], name, NC_NAME_LEN - 1) == 0) n = nc_counts[i];
  pthread_mutex_unlock(&nc_mu);
  return n;
}
int nvtx_pushes(void) {
  pthread_mutex_lock(&nc_mu);
  int n = 0;
  for (int i = 0; i < nc_n_names; ++i) n += nc_counts[i];
  pthread_mutex_unlock(&nc_mu);
  return n;
}
int nvtx_pops(void) { return nc_pops; }
int nvtx_unbalanced(void) { return nc_unbalanced; }
