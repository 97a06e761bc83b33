"""GB300-native forward-stable DPR1 eigensolver (arXiv 1405.7537).

The CUDA library is loaded on first use; see ``binding``.
"""
