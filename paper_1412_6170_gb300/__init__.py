"""GB300-native repeated k-NN over moving objects (arXiv 1412.6170 hot path).

The per-tick spatial join -- PR-quadtree rebuild, per-query expansion with a
top-k and the covered-disc check, result compaction -- runs as hand-written
sm_103a CUDA kernels behind the C-ABI declared in ``include/knn.h``.  This
package holds the ctypes binding of that library (``knnq``) and the seeded
synthetic workloads (``synth``).
"""
