"""GB300-native uniform-grid integration (density, local Hamiltonian, grid forces)
for numerical atomic orbitals."""
