/* Prints sizeof/offsetof of the public structs, compiled against include/ranc.h
 * by the ABI test so the Python binding's layout is checked against the C one. */
#include <stddef.h>
#include <stdio.h>
#include "ranc.h"
#define OFF(f) printf(#f " %zu\n", offsetof(ranc_desc, f))
int main(void)
{
    printf("sizeof_dest %zu\nsizeof_desc %zu\n", sizeof(ranc_dest), sizeof(ranc_desc));
    printf("dest.axon %zu\ndest.delay %zu\ndest.kind %zu\n", offsetof(ranc_dest, axon), offsetof(ranc_dest, delay),
           offsetof(ranc_dest, kind));
    OFF(grid_w); OFF(neg_mode); OFF(core_xy); OFF(crossbar); OFF(axon_type); OFF(weight); OFF(leak); OFF(pos_thr);
    OFF(neg_thr); OFF(reset); OFF(v0); OFF(dest); OFF(n_inputs); OFF(n_outputs); OFF(in_offsets); OFF(in_core);
    OFF(in_axon);
    return 0;
}
