"""FP64 CPU oracle of the Icarus 3.0 hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may import this
package. The CUDA library and its Python binding never use it.
"""
