"""pifepic-gb300: GB300-native hot path of the non-homogeneous IFE-PIC method
of arXiv:2011.10214 (PIFE-PIC).

  capi       ctypes binding of libpifepic (loads the CUDA library; raises if absent)
  build      compiles libpifepic.so for sm_103a in-tree
  workloads  seeded synthetic problem set-ups (no method arithmetic)
"""
