"""GB300-native spectral boundary-integral operators for N rigid spheres in
Stokes flow (Corona & Veerapaneni, arXiv:1707.06551).

The compute path is the CUDA library ``libsphere_bie.so`` (sm_103a) behind the
C interface of ``include/sphere_bie.h``; ``sphere_bie`` is its thin ctypes
binding.  ``workloads`` holds the seeded synthetic suspensions.  Importing the
package loads nothing; the library is loaded on first use of the binding and
a missing library raises instead of falling back to anything else.
"""
