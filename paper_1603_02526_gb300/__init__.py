"""GB300-native ADMM on a factor graph (Hao et al., "Testing fine-grained
parallelism for the ADMM on a factor-graph").

The solver is libfgadmm.so (include/fgadmm.h, CUDA for sm_103a); this
package holds its thin Python binding, the in-tree build step and the seeded
synthetic inputs.  Importing the package does not load the library; the
first binding call does, and fails loudly if it has not been built.
"""
__all__ = ["inputs", "graph", "build"]
