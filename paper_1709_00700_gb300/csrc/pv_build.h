// Build pipelines (Table 2): LOOP over a dimension, FILTER, HASH_PUT of the
// key with its payload into a linear-probing, cuckoo or perfect-array table.
#pragma once

#include <string>
#include <cuda_runtime.h>

#include "pv.h"
#include "pv_device.cuh"

namespace pv {

struct BuildInput {
  int64_t n_rows;                 // rows of the build table (an upper bound when n_dyn is set)
  const unsigned long long* n_dyn; // row count read on the device (an earlier pipeline's result), or null
  const void* key;
  int key_type;
  int n_preds;
  const void* pred_col[PV_MAX_PREDS];
  int pred_type[PV_MAX_PREDS];
  int64_t lo[PV_MAX_PREDS], hi[PV_MAX_PREDS];
  int n_payload;
  const void* pay_col[PV_MAX_PAYLOAD];
  int pay_type[PV_MAX_PAYLOAD];
};

struct BuildParams {
  BuildInput in;
  DevHT ht;
  int max_evictions;
  int32_t* err;
  unsigned long long* pay_stats;  // [2 * PV_MAX_PAYLOAD]: max code, min code of each payload column
};

struct BuildTable {
  DevHT ht{};
  int n_payload = 0;
  bool indexed = false;               // two or more payload columns: slots hold the build row
  const void* pay_col[PV_MAX_PAYLOAD]{};  // indexed tables gather their payloads from these columns
  int pay_type[PV_MAX_PAYLOAD]{};
  int64_t pay_min[PV_MAX_PAYLOAD]{};  // over the surviving rows (empty: min > max)
  int64_t pay_max[PV_MAX_PAYLOAD]{};
  void* mem = nullptr;
  size_t slot_bytes = 0;  // bytes of the slot array (rebuilds clear them)
  BuildParams bp{};       // the build pipeline, kept for rebuilds
};

struct BuildEnv {
  cudaStream_t stream;
  int sm_count;
  int32_t* err;
  int* launches;
  void* (*alloc)(size_t, void*);
  void* user;
};

// Allocates the table through env.alloc, enqueues the build and reads back the
// payload statistics (synchronising the stream).  Kernel-detected errors
// (duplicate key, full table, cuckoo cycle) land in env.err.
pv_status build_table(const BuildEnv& env, const BuildInput& in, const pv_ht_variant& var, int64_t kmin,
                      int64_t kmax, BuildTable& out, std::string& msg);

// Enqueues the build pipeline of an existing table again (clear, insert,
// duplicate check): no allocation, no synchronisation; the payload
// statistics of the first build are kept.
pv_status rebuild_table(const BuildEnv& env, const BuildTable& t);

}  // namespace pv
