"""Build-time process generator: Feynman diagrams, colour-flow expansion, evaluation
schedule and emission of the per-process CUDA code."""
