"""GB300-native hybrid thermal pseudopotential lattice Boltzmann boiling step."""
