"""GB300-native Fossen 6-DOF underwater-vehicle fleet stepper (MarineGym's hydrodynamics +
integrator hot path).  Importing the package loads nothing; the CUDA library is loaded on first
use and its absence raises."""
__version__ = "0.1.0"
