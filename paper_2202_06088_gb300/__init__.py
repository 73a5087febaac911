"""GB300-native VOctree renderer (NeuVV, Sec. 4.3 and Sec. 5.1).

Importing the package loads nothing native; ``paper_2202_06088_gb300.binding``
loads the CUDA library and fails loudly when it is missing.
"""
