"""GB300-native Monte Carlo for the Levy LIBOR model (Papapantoleon & Skovmand,
"Numerical Methods for the Levy LIBOR model").

The compute runs in ``liblll.so`` (CUDA for sm_103a behind a C ABI declared in
``include/lll.h``); :mod:`paper_1006_3340_gb300.lll` is the thin ctypes binding.
Importing this package does not load the library; the binding loads it on
first use and raises if it is missing.
"""
