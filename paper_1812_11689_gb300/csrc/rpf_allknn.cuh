// rpf_allknn.cuh -- the all-kNN launch sequence without its closing wait.
#pragma once

#include <cuda_runtime.h>

#include "rpf_internal.cuh"

// Enqueues the leaf tiles and the cross-tree merges of every group of trees
// of rpf_all_knn_dev on s and returns without waiting: no allocation, no
// synchronisation, no host read of device memory, so the sequence can be
// recorded into a CUDA graph.  Bounded device waits that give up set the
// forest's error word (f->d_err).  ws: running lists then per-tree lists
// (the layout of rpf_all_knn_dev).
int rpf_all_knn_enqueue(rpf_forest* f, int T, int K, int32_t* idx, float* dist, void* ws,
                        size_t ws_bytes, cudaStream_t s, uint2* keys);
