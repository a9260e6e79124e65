"""GB300-native phase-field lattice Boltzmann solver for N-phase flow."""
