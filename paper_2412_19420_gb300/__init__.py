"""GB300-native Boolean-matrix frequent-itemset miner (arXiv 2412.19420).

Submodules:
  fim      ctypes binding of libfim (include/fim.h) -- the product API
  build    compiles libfim.so for sm_103a
  datagen  seeded synthetic transaction databases (inputs only)
Importing the package loads nothing; import ``paper_2412_19420_gb300.fim``
for the miner (it raises if libfim.so is missing).
"""
